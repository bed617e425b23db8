"""Point sets unlike proteins: an SPH-like particle cloud with radii spread over a
factor of 8 (against about 1.2 for atoms), so neighbour counts vary from a few
to over a hundred and many atoms take the wide-row path of the per-atom kernel;
spreads of 12 and 16 reach 257..512 and 513..1,024 neighbours.
The whole complex must equal the oracle's, for alpha 0 and alpha > 0, in both
predicate modes.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_complex, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("alpha,mode", [(0.0, 0), (0.5, 0), (0.0, 1)], ids=["a0-filtered", "a0.5-filtered", "a0-fp64"])
def test_particles_equal_oracle(alpha, mode):
    c, r = synth.particles(11, 3000)
    gpu = run_gpu(c, r, alpha, precision=mode)
    st = gpu.stats()
    assert st["max_degree"] > 64, "the cloud should exercise the wide-row path"
    assert_same_complex(gpu, oracle.alpha_complex(c, r, alpha))


def test_particles_chunked_equal_whole():
    import paper_1908_05944_gb300 as ac

    c, r = synth.particles(12, 6000)
    whole = run_gpu(c, r, 0.0)
    ch = ac.ChunkedComplex(c, r, 0.0, 900)
    assert ch.stats()["n_chunks"] > 3
    for d in range(4):
        assert np.array_equal(ch.simplices(d), whole.simplices(d).cpu().numpy())
        assert np.array_equal(ch.filtration_values(d), whole.filtration_values(d).cpu().numpy())


def test_particles_beyond_256_neighbours():
    """Radii over a factor of 12: some particles have 257..512 grown-ball neighbours (the per-atom
    kernel's 512-entry rows, 10-bit row positions); the complex still equals the oracle's."""
    c, r = synth.particles(14, 3000, r_hi=3.0)
    gpu = run_gpu(c, r, 0.0)
    assert 256 < gpu.stats()["max_degree"] <= 512
    assert_same_complex(gpu, oracle.alpha_complex(c, r, 0.0))


def test_particles_beyond_512_neighbours():
    """Radii over a factor of 16: dozens of particles have 513..667 grown-ball neighbours and take the
    per-atom kernel's 32-word rows (working sets in global memory); the complex equals the oracle's."""
    c, r = synth.particles(14, 3000, r_hi=4.0)
    for mode in (0, 1):
        gpu = run_gpu(c, r, 0.0, precision=mode)
        assert 512 < gpu.stats()["max_degree"] <= 1024
        assert_same_complex(gpu, oracle.alpha_complex(c, r, 0.0))


def test_particles_candidate_lists_all_tiers():
    """The candidate lists (Sigma_ortho^1..3, the keep_candidates build) of a cloud whose particles
    reach every row width of the per-atom pass: up to 64 neighbours (shared-memory working sets),
    65..128, 129..256, 257..512 and 513..1,024 (working sets in global memory), against the oracle's."""
    c, r = synth.particles(14, 3000, r_hi=4.0)
    # grown-ball neighbour counts at alpha = 0 (balls meet: |c_i - c_x| <= r_i + r_x), in FP64: only
    # to show that every width is reached
    cc, rr = np.asarray(c, np.float64), np.asarray(r, np.float64)
    d2 = ((cc[:, None, :] - cc[None, :, :]) ** 2).sum(-1)
    deg = (d2 <= (rr[:, None] + rr[None, :]) ** 2).sum(1) - 1
    for lo, hi in ((1, 64), (65, 128), (129, 256), (257, 512), (513, 1024)):
        assert np.any((deg >= lo) & (deg <= hi)), (lo, hi)
    ref = oracle.alpha_complex(c, r, 0.0)
    gpu = run_gpu(c, r, 0.0, keep_candidates=True)
    assert gpu.stats()["max_degree"] > 512
    for d in (1, 2, 3):
        got = gpu.candidates(d).cpu().numpy()
        assert np.array_equal(got, ref.candidates[d]), f"Sigma_ortho^{d} differs"
    assert_same_complex(gpu, ref)


def test_particles_beyond_1024_neighbours_refused():
    import paper_1908_05944_gb300 as ac

    c, r = synth.particles(14, 4000, spacing=0.55, r_hi=4.0)  # denser: over 1,024 neighbours
    with pytest.raises(ac.AlphacError) as e:
        run_gpu(c, r, 0.0)
    assert e.value.code == ac.AC_ERR_CAPACITY and "at most 1024" in str(e.value)
