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


def test_particles_beyond_1024_neighbours_refused():
    import paper_1908_05944_gb300 as ac

    c, r = synth.particles(14, 4000, spacing=0.55, r_hi=4.0)  # denser: over 1,024 neighbours
    with pytest.raises(ac.AlphacError) as e:
        run_gpu(c, r, 0.0)
    assert e.value.code == ac.AC_ERR_CAPACITY and "at most 1024" in str(e.value)
