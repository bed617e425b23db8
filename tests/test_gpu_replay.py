"""Rebuilds of a context as a CUDA-graph replay.

The first ac_build of a context reads each list size back to the host; later
builds replay the same launches as one graph with those sizes checked on the
device. These tests check that a replayed build returns exactly what the
synchronised one did (and what the oracle does), that it waits on the host
fewer times, and that opt.no_graph keeps every build synchronised.
"""
import numpy as np
import pytest

import synth
from gpu_util import assert_same_complex

pytestmark = pytest.mark.gpu


def _snapshot(cx, mol=-1):
    out = []
    for d in range(4):
        out.append((cx.simplices(d, mol).cpu().numpy(), cx.attached(d, mol).cpu().numpy(),
                    cx.filtration_values(d, mol).cpu().numpy()))
    return out


def _assert_identical(a, b):
    for d in range(4):
        for x, y in zip(a[d], b[d]):
            assert x.shape == y.shape and np.array_equal(x, y), f"dim {d} differs between builds"


@pytest.mark.parametrize("precision", ["filtered", "plain_fp64"])
def test_replay_equals_first_build_and_oracle(precision):
    import torch

    import oracle
    import paper_1908_05944_gb300 as ac

    c, r = synth.workload("globule2k_vdw")
    p = ac.AC_PRECISION_FILTERED if precision == "filtered" else ac.AC_PRECISION_PLAIN_FP64
    cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0, ac.options(precision=p))
    cx.build()
    first = _snapshot(cx)
    st0 = cx.stats()
    assert st0["replayed"] == 0
    for _ in range(3):
        cx.build()
        st = cx.stats()
        assert st["replayed"] == 1
        assert st["host_syncs"] < st0["host_syncs"]
        assert st["simplices"] == st0["simplices"]
        _assert_identical(first, _snapshot(cx))
    assert_same_complex(cx, oracle.alpha_complex(c, r, 0.0))


def test_replay_on_another_stream():
    import torch

    import paper_1908_05944_gb300 as ac

    c, r = synth.workload("globule2k_vdw")
    cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0)
    cx.build()
    first = _snapshot(cx)
    side = torch.cuda.Stream()
    cx.build(side)
    cx.build(side)
    torch.cuda.synchronize()
    assert cx.stats()["replayed"] == 1
    _assert_identical(first, _snapshot(cx))


def test_no_graph_keeps_builds_synchronised():
    import torch

    import paper_1908_05944_gb300 as ac

    c, r = synth.workload("globule2k_vdw")
    cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0, ac.options(no_graph=True))
    cx.build()
    first = _snapshot(cx)
    cx.build()
    assert cx.stats()["replayed"] == 0
    _assert_identical(first, _snapshot(cx))


def test_batch_and_candidate_lists_replay():
    import torch

    import paper_1908_05944_gb300 as ac

    sizes = [300, 0, 1200, 57]
    mols = [synth.globule(2000 + m, n, probe=True) if n else (np.zeros((0, 3)), np.zeros(0))
            for m, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    c = torch.from_numpy(np.concatenate([m[0] for m in mols])).cuda()
    r = torch.from_numpy(np.concatenate([m[1] for m in mols])).cuda()
    bx = ac.AlphaComplex(c, r, 0.0, offsets=offsets)
    bx.build()
    first = [_snapshot(bx, m) for m in range(len(sizes))]
    bx.build()
    bx.build()
    assert bx.stats()["replayed"] == 1
    for m in range(len(sizes)):
        _assert_identical(first[m], _snapshot(bx, m))

    c1, r1 = synth.workload("globule2k_vdw")
    kx = ac.AlphaComplex(torch.from_numpy(c1).cuda(), torch.from_numpy(r1).cuda(), 0.0,
                         ac.options(keep_candidates=True))
    kx.build()
    cand = [kx.candidates(d).cpu().numpy() for d in (1, 2, 3)]
    kx.build()
    assert kx.stats()["replayed"] == 1
    for d, want in zip((1, 2, 3), cand):
        assert np.array_equal(kx.candidates(d).cpu().numpy(), want)


def test_host_results_equal_device_lists():
    """opt.host_results: the build copies each list to page-locked host memory as soon as it is
    final; the copies equal the device lists, after the first build and after replays, per molecule."""
    import torch

    import paper_1908_05944_gb300 as ac

    c, r = synth.workload("globule2k_vdw")
    for filtration in (ac.AC_FILTRATION_SIZE, ac.AC_FILTRATION_ORTHOSIZE):
        cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0,
                             ac.options(host_results=True, filtration=filtration))
        for _ in range(3):
            cx.build()
            for d in range(4):
                t, f, a = cx.host_lists(d)
                assert np.array_equal(t, cx.simplices(d).cpu().numpy())
                assert np.array_equal(f, cx.filtration_values(d).cpu().numpy())
                assert np.array_equal(a, cx.attached(d).cpu().numpy())
        assert cx.stats()["replayed"] == 1
    sizes = [300, 0, 800]
    mols = [synth.globule(2100 + m, n, probe=True) if n else (np.zeros((0, 3)), np.zeros(0))
            for m, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    bx = ac.AlphaComplex(torch.from_numpy(np.concatenate([m[0] for m in mols])).cuda(),
                         torch.from_numpy(np.concatenate([m[1] for m in mols])).cuda(), 0.0, ac.options(host_results=True),
                         offsets=offsets)
    bx.build()
    for m in range(len(sizes)):
        for d in range(4):
            t, f, a = bx.host_lists(d, m)
            assert np.array_equal(t, bx.simplices(d, m).cpu().numpy())
            assert np.array_equal(f, bx.filtration_values(d, m).cpu().numpy())
    plain = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0).build()
    with pytest.raises(ac.AlphacError) as e:
        plain.host_lists(1)
    assert e.value.code == ac.AC_ERR_STATE
