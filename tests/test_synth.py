"""The seeded input generator: deterministic, and the shape of the stated recipe."""
import numpy as np

import synth


def test_deterministic_and_seed_dependent():
    a = synth.globule(11, 500)
    b = synth.globule(11, 500)
    c = synth.globule(12, 500)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])


def test_recipe_properties():
    n = 5000
    xyz, rad, el = synth.atoms_int(3, n, synth.ball_radius(n), -1.0, probe=True)
    # minimum separation 1.3 A (integer squared distance >= ceil((1.3*1024)^2))
    from scipy.spatial import cKDTree
    d, _ = cKDTree(xyz.astype(np.float64)).query(xyz.astype(np.float64), k=2)
    assert (d[:, 1] ** 2).min() >= 1772094 - 1e-6
    # inside the ball (tested before quantisation: allow half a quantum per axis)
    R = synth.ball_radius(n) * 1024
    assert np.sqrt((xyz.astype(np.float64) ** 2).sum(1)).max() <= R + 1.0
    # element mix C .63, N .17, O .19, S .01 and the probe radii
    frac = np.bincount(el, minlength=4) / n
    assert np.allclose(frac, [0.63, 0.17, 0.19, 0.01], atol=0.02)
    assert set(np.unique(rad)) <= {3174, 3021, 2990, 3277}
    c, r = synth.globule(3, 100, probe=False)
    assert set(np.unique(np.rint(r * 1024).astype(int))) <= {1741, 1587, 1556, 1843}
    assert np.array_equal(c * 1024, np.rint(c * 1024))


def test_shell_and_batch_sizes():
    xyz, _, _ = synth.atoms_int(3, 20000, 361.0, 320.0)
    rr = np.sqrt((xyz.astype(np.float64) ** 2).sum(1)) / 1024
    assert rr.min() >= 320.0 - 1e-3 and rr.max() <= 361.0 + 1e-3
    s = synth.batch_sizes(4, 1024)
    assert s.min() >= 500 and s.max() <= 50000
    assert 9e6 < s.sum() < 1.3e7
    # log-uniform: the median sits near the geometric mean sqrt(500 * 50000) = 5000
    assert 3500 < np.median(s) < 7000


def test_normal_draws():
    w = synth.normal(6, 100001)
    assert abs(w.mean()) < 0.02 and abs(w.std() - 1) < 0.02


def test_particles_generator():
    """The SPH-like cloud: seeded, exact multiples of 1/1024, distinct centres, radii in range."""
    c, r = synth.particles(11, 5000)
    c2, r2 = synth.particles(11, 5000)
    assert np.array_equal(c, c2) and np.array_equal(r, r2)
    assert not np.array_equal(c, synth.particles(12, 5000)[0])
    q = c * 1024.0
    assert np.array_equal(q, np.round(q)) and np.array_equal(r * 1024.0, np.round(r * 1024.0))
    assert len(np.unique(np.round(q).astype(np.int64), axis=0)) == len(c)
    assert r.min() >= 0.25 and r.max() <= 2.0 and r.max() / r.min() > 7.0
