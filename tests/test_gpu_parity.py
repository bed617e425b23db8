"""CUDA path vs the exact oracle, element by element (simplex lists bit-exact, values 1e-12 relative).

Covers the small workload (2,000 atoms, van der Waals radii), probe-radius
globules that span many grid cells, both predicate modes, the estimation-pass
lists (Sigma_ortho^1..3, Step 1), the hand-derived fixtures, ties on lattices
(symbolic perturbation), empty and tiny inputs, one-cell inputs, atoms on cell
boundaries, far-off coordinates, alpha > 0 and alpha < 0, and error codes.
"""
import numpy as np
import pytest

import oracle
import synth
from golden_io import fixtures, read_fixture
from gpu_util import assert_same_complex, run_gpu

pytestmark = pytest.mark.gpu

MODES = {"filtered": 0, "plain_fp64": 1}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import importlib

    importlib.import_module("paper_1908_05944_gb300.build").build()


@pytest.mark.parametrize("mode", MODES)
def test_globule2k_vdw(mode):
    c, r = synth.workload("globule2k_vdw")
    ref = oracle.alpha_complex(c, r, 0.0)
    gpu = run_gpu(c, r, 0.0, precision=MODES[mode])
    assert_same_complex(gpu, ref)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed,n", [(11, 1500), (12, 4000), (13, 6321)])
def test_probe_globules(mode, seed, n):
    c, r = synth.globule(seed, n, probe=True)
    ref = oracle.alpha_complex(c, r, 0.0)
    gpu = run_gpu(c, r, 0.0, precision=MODES[mode])
    assert_same_complex(gpu, ref)


@pytest.mark.parametrize("probe", [False, True])
def test_estimation_lists_equal_sigma_ortho(probe):
    c, r = synth.globule(21, 3000, probe=probe)
    ref = oracle.alpha_complex(c, r, 0.0)
    gpu = run_gpu(c, r, 0.0, keep_candidates=True)
    for d in (1, 2, 3):
        got = gpu.candidates(d).cpu().numpy()
        assert np.array_equal(got, ref.candidates[d]), f"Sigma_ortho^{d} differs"
    st = gpu.stats()
    assert st["candidates"][1:] == [len(ref.candidates[d]) for d in (1, 2, 3)]
    assert_same_complex(gpu, ref)


@pytest.mark.parametrize("path", fixtures(), ids=lambda p: p.rsplit("/", 1)[-1])
def test_golden_fixtures(path):
    atoms, alpha, expect = read_fixture(path)
    if alpha is None:
        pytest.skip("alpha = infinity is an oracle-only mode")
    c = np.array([[float(a[0]), float(a[1]), float(a[2])] for a in atoms])
    r = np.array([float(a[3]) for a in atoms])
    if float(r.max()) ** 2 + float(alpha) > 16.0:
        # beyond the library's exact-integer range (r_max^2 + alpha <= 16 A^2): refused, not wrong
        import paper_1908_05944_gb300 as ac

        with pytest.raises(ac.AlphacError) as e:
            run_gpu(c, r, float(alpha))
        assert e.value.code == ac.AC_ERR_RANGE
        return
    gpu = run_gpu(c, r, float(alpha))
    got = {}
    for d in range(4):
        s = gpu.simplices(d).cpu().numpy()
        f = gpu.filtration_values(d).cpu().numpy()
        a = gpu.attached(d).cpu().numpy()
        for i, t in enumerate(s):
            got[tuple(int(x) for x in t)] = (f[i], bool(a[i]))
    assert set(got) == set(expect)
    for t, (f, att) in expect.items():
        assert got[t][1] == att
        assert got[t][0] == pytest.approx(float(f), rel=1e-14, abs=0)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", range(6))
def test_lattice_ties(mode, seed):
    """Many exact ties: co-orthospherical, coplanar and collinear subsets."""
    rng = np.random.default_rng(seed)
    n = 60 + 20 * seed
    pts = set()
    while len(pts) < n:
        pts.add(tuple(int(v) for v in rng.integers(-3, 4, 3)))
    pts = sorted(pts, key=lambda p: rng.random())
    spacing = 1.5 if seed % 2 else 2.0
    c = np.array(pts, dtype=np.float64) * spacing
    radii_choices = np.array([1.25, 1.5]) if seed % 3 else np.array([1.5])
    r = rng.choice(radii_choices, n)
    for alpha in (0.0, 0.5):
        ref = oracle.alpha_complex(c, r, alpha)
        gpu = run_gpu(c, r, alpha, precision=MODES[mode])
        assert_same_complex(gpu, ref)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 7])
def test_tiny_inputs(n):
    c, r = synth.globule(30 + n, max(n, 1), probe=True)
    c, r = c[:n], r[:n]
    ref = oracle.alpha_complex(c, r, 0.0)
    gpu = run_gpu(c, r, 0.0)
    assert_same_complex(gpu, ref)


@pytest.mark.parametrize("mode", MODES)
def test_halfway_quantisation(mode):
    # centres and radii halfway between two quanta round half to even on both sides:
    # a pair of equal balls 2048.5 quanta apart is an edge of Size exactly 0 at alpha = 0,
    # 2049.5 quanta apart it is not; radii 1000.5 and 1001.5 quanta give R = 1000 and 1002
    q = 1024.0
    c = np.array([[0.0, 0.0, 0.0], [2048.5 / q, 0.0, 0.0], [40.0, 0.0, 0.0], [40.0 - 2049.5 / q, 0.0, 0.0],
                  [0.0, 40.0, 0.0], [0.0, -40.0, 0.0], [0.0, 0.0, -2048.5 / q]])
    r = np.array([1.0, 1.0, 1.0, 1.0, 1000.5 / q, 1001.5 / q, 1.0])
    ref = oracle.alpha_complex(c, r, 0.0)
    gpu = run_gpu(c, r, 0.0, precision=MODES[mode])
    assert_same_complex(gpu, ref)
    assert gpu.simplices(1).cpu().numpy().tolist() == [[0, 1], [0, 6]]
    assert gpu.filtration_values(1).cpu().numpy().tolist() == [0.0, 0.0]
    f0 = gpu.filtration_values(0).cpu().numpy()
    assert f0[4] == -(1000 * 1000) / 2.0**20 and f0[5] == -(1002 * 1002) / 2.0**20
    # alpha halfway between two quanta: equal balls 2050 quanta apart have edge Size 2049 / 2^20;
    # alpha 2048.5 / 2^20 rounds to 2048 (no edge), 2049.5 / 2^20 to 2050 (edge)
    c2 = np.array([[0.0, 0.0, 0.0], [2050.0 / q, 0.0, 0.0]])
    for a_half, edges in ((2048.5, 0), (2049.5, 1)):
        alpha = a_half / 2.0**20
        ref = oracle.alpha_complex(c2, np.ones(2), alpha)
        gpu = run_gpu(c2, np.ones(2), alpha, precision=MODES[mode])
        assert_same_complex(gpu, ref)
        assert gpu.count(1) == edges


def test_all_atoms_in_one_cell():
    rng = np.random.default_rng(5)
    c = np.round(rng.uniform(0, 1.5, (12, 3)) * 1024) / 1024
    r = np.full(12, 3.0)
    ref = oracle.alpha_complex(c, r, 0.0)
    assert_same_complex(run_gpu(c, r, 0.0), ref)


def test_atoms_on_cell_boundaries():
    # cell side = ceil(1024 * sqrt(r_max^2 + alpha)) quanta; put centres on multiples of it
    r0 = 1.5
    side = np.ceil(1024 * r0) / 1024
    g = np.arange(-3, 4) * side
    c = np.array([[x, y, z] for x in g for y in g for z in g[:3]])
    r = np.full(len(c), r0)
    ref = oracle.alpha_complex(c, r, 0.0)
    assert_same_complex(run_gpu(c, r, 0.0), ref)


def test_far_coordinates_and_translation():
    c, r = synth.globule(41, 1200, probe=True)
    ref = oracle.alpha_complex(c, r, 0.0)
    shifted = c + np.array([100000.0, -250000.0, 31337.0])
    assert_same_complex(run_gpu(shifted, r, 0.0), ref)


@pytest.mark.parametrize("alpha", [1.4, 2.0, -1.0])
def test_other_alphas(alpha):
    c, r = synth.globule(51, 2500, probe=alpha < 0)
    if alpha > 0:
        r = np.minimum(r, 2.0)  # keep r_max^2 + alpha within 16 A^2
    ref = oracle.alpha_complex(c, r, alpha)
    assert_same_complex(run_gpu(c, r, alpha), ref)


def test_coordinate_range_limits():
    """Two clusters centred at x = -(2^20 - 16) A and +(2^20 - 16) A (quantised coordinates just below
    2^30 in magnitude, the extremes less than 2^31 apart) build and equal the oracle; a coordinate that
    rounds to 2^30 quanta is refused."""
    import paper_1908_05944_gb300 as ac

    parts = []
    for k, sx in enumerate((-1.0, 1.0)):
        c, r = synth.globule(80 + k, 120, probe=True)
        parts.append((c + np.array([sx * 1048560.0, 0.0, 0.0]), r))
    c = np.concatenate([p[0] for p in parts])
    r = np.concatenate([p[1] for p in parts])
    assert np.abs(np.rint(c * 1024)).max() < 2**30
    assert_same_complex(run_gpu(c, r, 0.0), oracle.alpha_complex(c, r, 0.0))
    for edge in (1048576.0, -1048576.0, 1048576.0 - 1.0 / 4096.0):
        bad = c.copy()
        bad[5, 1] = edge
        with pytest.raises(ac.AlphacError) as e:
            run_gpu(bad, r, 0.0)
        assert e.value.code == ac.AC_ERR_RANGE


def test_error_codes():
    import paper_1908_05944_gb300 as ac

    c = np.zeros((2, 3))
    r = np.ones(2)
    with pytest.raises(ac.AlphacError) as e:
        run_gpu(c, r)
    assert e.value.code == ac.AC_ERR_DEGENERATE
    with pytest.raises(ac.AlphacError) as e:
        run_gpu(np.array([[np.nan, 0, 0]]), np.ones(1))
    assert e.value.code == ac.AC_ERR_INVALID_ARG
    with pytest.raises(ac.AlphacError) as e:
        run_gpu(np.zeros((1, 3)), np.array([-1.0]))
    assert e.value.code == ac.AC_ERR_INVALID_ARG
    with pytest.raises(ac.AlphacError) as e:
        run_gpu(np.zeros((1, 3)), np.array([4.5]))
    assert e.value.code == ac.AC_ERR_RANGE
    with pytest.raises(ac.AlphacError) as e:
        run_gpu(np.zeros((1, 3)), np.array([3.5]), alpha=5.0)
    assert e.value.code == ac.AC_ERR_RANGE


def test_results_before_build_are_refused():
    import torch

    import paper_1908_05944_gb300 as ac

    cx = ac.AlphaComplex(torch.zeros((1, 3), dtype=torch.float64).cuda(), torch.ones(1, dtype=torch.float64).cuda())
    with pytest.raises(ac.AlphacError) as e:
        cx.simplices(0)
    assert e.value.code == ac.AC_ERR_STATE


def test_rebuild_is_deterministic():
    c, r = synth.globule(61, 3000, probe=True)
    gpu = run_gpu(c, r, 0.0)
    first = [gpu.simplices(d).cpu().numpy() for d in range(4)]
    fv = [gpu.filtration_values(d).cpu().numpy() for d in range(4)]
    gpu.build()
    for d in range(4):
        assert np.array_equal(first[d], gpu.simplices(d).cpu().numpy())
        assert np.array_equal(fv[d], gpu.filtration_values(d).cpu().numpy())


@pytest.mark.parametrize("k", [250, 400])
def test_star_with_oversized_buckets(k):
    """Atom 0 at the centre of k atoms on a sphere: 2k - 4 tetrahedra, 3k - 6 triangles and k edges share
    their first vertex, beyond one warp's sort (256 items), and atom 0 has k neighbours (wide rows: 256
    entries for k = 250, 512 for k = 400)."""
    i = np.arange(k) + 0.5
    phi = np.arccos(1 - 2 * i / k)
    th = np.pi * (1 + 5 ** 0.5) * i
    pts = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1) * 2.0
    c = np.vstack([[0.0, 0.0, 0.0], pts])
    r = np.full(len(c), 1.0)
    r[0] = 1.6
    ref = oracle.alpha_complex(c, r, 0.5)
    assert (ref.simplices[3][:, 0] == 0).sum() > 256
    gpu = run_gpu(c, r, 0.5)
    assert_same_complex(gpu, ref)
    gpu.build()  # and its replay
    assert_same_complex(gpu, ref)


def test_sparse_clusters_coarse_grid():
    """Eight clusters at the corners of a 20,000 A cube: the dense cell table is coarsened until the
    cells are far wider than 2h, and the neighbour search takes its 64-bit path."""
    parts = []
    for k in range(8):
        c, r = synth.globule(70 + k, 150, probe=True)
        corner = np.array([(k >> 0) & 1, (k >> 1) & 1, (k >> 2) & 1]) * 20000.0
        parts.append((c + corner, r))
    c = np.concatenate([p[0] for p in parts])
    r = np.concatenate([p[1] for p in parts])
    ref = oracle.alpha_complex(c, r, 0.0)
    gpu = run_gpu(c, r, 0.0)
    assert_same_complex(gpu, ref)
    dims = gpu.stats()["grid_dims"]
    assert max(dims) < 400  # cells over 37,837 quanta wide (about 6,000 cells per axis uncoarsened)
