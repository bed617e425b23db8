"""The bounded wait of the single-pass scan, made to run out on purpose.

Scans of more than 4 M elements (list offsets) are single-pass: each tile of
4,096 elements waits for the sums of the tiles before it. The wait is bounded;
ALPHAC_SCAN_SPIN_LIMIT < 0 makes every tile give up once. A tile that gives up
adds the missing sum from the inputs itself, so the build's lists stay exact,
while ac_build reports AC_ERR_TIMEOUT. No kernel faults, traps or hangs here:
the wait ends by its count, and the error comes back as a status.

* A sparse cloud (200,000 atoms in a 540 A cube) has about 5.8 M grid cells,
  so the scan of the cell offsets takes the single-pass path.
* The 1,024-molecule batch (10.7 M atoms) takes it for the per-atom offsets
  too, among them in-place scans (input and output the same array).
After the failed call, a build of the same context with the default limit
equals a build that never timed out.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _same(a, b):
    mols = [-1] if a.n_mol == 1 else range(a.n_mol)
    for m in mols:
        for d in range(4):
            assert np.array_equal(a.simplices(d, m).cpu().numpy(), b.simplices(d, m).cpu().numpy()), (m, d)
            assert np.array_equal(a.attached(d, m).cpu().numpy(), b.attached(d, m).cpu().numpy()), (m, d)
            assert np.array_equal(a.filtration_values(d, m).cpu().numpy(),
                                  b.filtration_values(d, m).cpu().numpy()), (m, d)


def _timeout_then_rebuild(monkeypatch, make):
    import paper_1908_05944_gb300 as ac

    ref = make(ac.options()).build()
    monkeypatch.setenv("ALPHAC_SCAN_SPIN_LIMIT", "-1")
    cx = make(ac.options(no_graph=True))
    with pytest.raises(ac.AlphacError) as e:
        cx.build()
    assert e.value.code == ac.AC_ERR_TIMEOUT
    monkeypatch.delenv("ALPHAC_SCAN_SPIN_LIMIT")
    cx.build()
    _same(cx, ref)
    return cx


def test_sparse_cloud_grid_scan(monkeypatch):
    import torch

    import oracle
    import paper_1908_05944_gb300 as ac

    rng = np.random.default_rng(11)
    c = np.round(rng.uniform(-270.0, 270.0, (200000, 3)) * 1024.0) / 1024.0
    r = np.round(rng.uniform(1.0, 1.5, 200000) * 1024.0) / 1024.0
    assert len(np.unique(c, axis=0)) == len(c)
    tc, tr = torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda()
    cx = _timeout_then_rebuild(monkeypatch, lambda o: ac.AlphaComplex(tc, tr, 0.0, o))
    grid = cx.stats()["grid_dims"]
    assert grid[0] * grid[1] * grid[2] > 4 * 1024 * 1024  # the single-pass scan ran
    from gpu_util import assert_same_complex

    assert_same_complex(cx, oracle.alpha_complex(c, r, 0.0))


def test_batch_per_atom_scans(monkeypatch):
    import torch

    import paper_1908_05944_gb300 as ac

    mols = synth.batch()
    offsets = np.concatenate([[0], np.cumsum([len(r) for _, r in mols])])
    assert offsets[-1] > 4 * 1024 * 1024
    c_all = torch.from_numpy(np.concatenate([m[0] for m in mols])).cuda()
    r_all = torch.from_numpy(np.concatenate([m[1] for m in mols])).cuda()
    cx = _timeout_then_rebuild(monkeypatch, lambda o: ac.AlphaComplex(c_all, r_all, 0.0, o, offsets=offsets))
    assert cx.stats()["simplices"][0] > 4 * 1024 * 1024
