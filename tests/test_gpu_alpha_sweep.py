"""The alpha sweep: sub-complexes of a built filtration at smaller alphas.

K_alpha2 = {sigma in K_alpha : Size(sigma) <= alpha2} (Section 2.4); the GPU
decides it exactly on the rational Size. Each sub-complex must equal the
oracle's complex built directly at alpha2, rows and values.
"""
import numpy as np
import pytest

import synth
from gpu_util import assert_values

pytestmark = pytest.mark.gpu


def _check_sub(cx, ref, alpha2):
    sub = cx.subcomplex(alpha2)
    for d in range(4):
        got = sub[d][0].cpu().numpy()
        want = ref.simplices[d]
        assert got.shape == want.shape, f"alpha2={alpha2} dim {d}: {got.shape[0]} vs {want.shape[0]}"
        assert np.array_equal(got, want), f"alpha2={alpha2} dim {d}: rows differ"
        assert_values(sub[d][1].cpu().numpy(), ref.f[d], f"alpha2={alpha2} dim {d}")


@pytest.mark.parametrize("workload,alpha,alphas2", [
    ("vdw", 1.5, [-0.5, 0.0, 0.37, 0.9, 1.5]),
    ("probe", 2.0, [0.0, 0.25, 1.0, 2.0]),
])
def test_subcomplex_equals_direct_build(workload, alpha, alphas2):
    import torch

    import oracle
    import paper_1908_05944_gb300 as ac

    if workload == "vdw":
        c, r = synth.workload("globule2k_vdw")
    else:
        c, r = synth.globule(71, 3000, probe=True)
    cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), alpha).build()
    for a2 in alphas2:
        _check_sub(cx, oracle.alpha_complex(c, r, a2), a2)


def test_subcomplex_at_a_tie():
    """alpha2 exactly at an attained Size keeps that simplex (inclusive), on lattice inputs full of ties."""
    import torch

    import oracle
    import paper_1908_05944_gb300 as ac

    g = np.arange(4, dtype=np.float64) * 1.5
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    r = np.full(len(c), 1.0)
    cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 2.0).build()
    f1 = cx.filtration_values(1).cpu().numpy()
    vals = np.unique(f1[(f1 > -1.0) & (f1 < 2.0)])
    for a2 in vals[:: max(1, len(vals) // 4)]:
        _check_sub(cx, oracle.alpha_complex(c, r, float(a2)), float(a2))


def test_subcomplex_arguments():
    import torch

    import paper_1908_05944_gb300 as ac

    c, r = synth.workload("globule2k_vdw")
    cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.5).build()
    with pytest.raises(ac.AlphacError) as e:
        cx.subcomplex_mask(1, 0.75)
    assert e.value.code == ac.AC_ERR_INVALID_ARG
    mask, n = cx.subcomplex_mask(2, 0.5)
    assert n == cx.count(2) and bool(mask.all())
