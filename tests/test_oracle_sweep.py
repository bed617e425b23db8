"""Oracle pin: the filtration values are a filtration of the alpha complexes.

For alpha2 <= alpha, the complex built at alpha2 is exactly the set of
simplices of the complex at alpha whose value (Size) is <= alpha2 (Section
2.4), in the same order. alpha2 is taken between consecutive distinct values,
away from every value, so the FP64 rounding of the values cannot decide it.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("seed,n,probe,alpha", [(81, 400, False, 1.5), (82, 600, True, 2.0)])
def test_complex_at_smaller_alpha_is_a_sublevel_set(seed, n, probe, alpha):
    c, r = synth.globule(seed, n, probe=probe)
    big = oracle.alpha_complex(c, r, alpha)
    vals = np.unique(np.concatenate([f for f in big.f]))
    gaps = np.nonzero(np.diff(vals) > 1e-6 * np.maximum(1.0, np.abs(vals[1:])))[0]
    picks = gaps[np.linspace(0, len(gaps) - 1, 6).astype(int)]
    for k in picks:
        a2 = float(np.round((vals[k] + vals[k + 1]) / 2 * 2**20) / 2**20)  # quantised like alpha
        small = oracle.alpha_complex(c, r, a2)
        for d in range(4):
            keep = big.f[d] <= a2
            assert np.array_equal(big.simplices[d][keep], small.simplices[d]), f"alpha2={a2} dim {d}"
            assert np.array_equal(big.f[d][keep], small.f[d]), f"alpha2={a2} dim {d} values"
