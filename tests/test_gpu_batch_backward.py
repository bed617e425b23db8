"""Batched contexts and the FP64 backward.

* A batch of molecules built in one context equals the single-molecule builds
  and the oracle, molecule by molecule.
* Backward (combinatorics fixed): against the oracle's closed-form gradient
  and against central differences of ac_eval_filtration (step 1e-6 A, 64
  random centre coordinates and 64 random radii, relative error <= 1e-6) on
  the 20,000-atom globule; repeated calls give bit-identical gradients.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_complex, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_batch_equals_single_and_oracle():
    import torch

    import paper_1908_05944_gb300 as ac

    sizes = synth.batch_sizes(4, 1024)[:12]
    mols = [synth.globule(1000 + m, int(n), probe=True) for m, n in enumerate(sizes)]
    mols.insert(3, (np.zeros((0, 3)), np.zeros(0)))  # an empty molecule
    offsets = np.concatenate([[0], np.cumsum([len(r) for _, r in mols])])
    c = np.concatenate([m[0] for m in mols])
    r = np.concatenate([m[1] for m in mols])
    batch = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0, offsets=offsets).build()
    for m, (cm, rm) in enumerate(mols):
        ref = oracle.alpha_complex(cm, rm, 0.0)
        assert_same_complex(batch, ref, mol=m)
        if len(rm):
            single = run_gpu(cm, rm, 0.0)
            for d in range(4):
                assert np.array_equal(single.simplices(d).cpu().numpy(), batch.simplices(d, m).cpu().numpy())


@pytest.fixture(scope="module")
def globule20k():
    import torch

    c, r = synth.workload("globule20k_probe")
    gpu = run_gpu(c, r, 0.0)
    ref = oracle.alpha_complex(c, r, 0.0)
    counts = [gpu.count(d) for d in range(4)]
    w_all = synth.normal(synth.LOSS_WEIGHT_SEED, sum(counts))
    w, k = [], 0
    for d in range(4):
        w.append(w_all[k:k + counts[d]])
        k += counts[d]
    wt = [torch.from_numpy(x).cuda() for x in w]
    return c, r, gpu, ref, w, wt


def test_backward_matches_closed_form(globule20k):
    c, r, gpu, ref, w, wt = globule20k
    assert_same_complex(gpu, ref)
    dc, dr = gpu.backward(wt)
    oc, orr = ref.gradient(w)
    dc, dr = dc.cpu().numpy(), dr.cpu().numpy()
    scale_c = np.abs(oc).max()
    scale_r = np.abs(orr).max()
    assert np.max(np.abs(dc - oc)) <= 1e-9 * scale_c
    assert np.max(np.abs(dr - orr)) <= 1e-9 * scale_r


def test_backward_matches_finite_differences(globule20k):
    import torch

    c, r, gpu, ref, w, wt = globule20k
    dc, dr = gpu.backward(wt)
    dc = dc.cpu().numpy()
    rng = np.random.default_rng(64)
    h = 1e-6
    ct = torch.from_numpy(c).cuda()
    rt = torch.from_numpy(r).cuda()
    atoms = rng.choice(len(r), 64, replace=False)
    axes = rng.integers(0, 3, 64)
    for a, ax in zip(atoms, axes):
        cp = ct.clone()
        cm = ct.clone()
        cp[a, ax] += h
        cm[a, ax] -= h
        fp = gpu.eval_filtration(cp, rt)
        fm = gpu.eval_filtration(cm, rt)
        g = 0.0
        for d in range(4):
            diff = (fp[d] - fm[d]).cpu().numpy()
            g += float(np.dot(w[d], diff))
        g /= 2 * h
        assert abs(g - dc[a, ax]) <= 1e-6 * max(abs(dc[a, ax]), 1e-3), (a, ax, g, dc[a, ax])


def test_backward_radii_match_finite_differences(globule20k):
    import torch

    c, r, gpu, ref, w, wt = globule20k
    _, dr = gpu.backward(wt)
    dr = dr.cpu().numpy()
    rng = np.random.default_rng(65)
    h = 1e-6
    ct = torch.from_numpy(c).cuda()
    rt = torch.from_numpy(r).cuda()
    for a in rng.choice(len(r), 64, replace=False):
        rp = rt.clone()
        rm = rt.clone()
        rp[a] += h
        rm[a] -= h
        fp = gpu.eval_filtration(ct, rp)
        fm = gpu.eval_filtration(ct, rm)
        g = sum(float(np.dot(w[d], (fp[d] - fm[d]).cpu().numpy())) for d in range(4)) / (2 * h)
        assert abs(g - dr[a]) <= 1e-6 * max(abs(dr[a]), 1e-3), (a, g, dr[a])


def test_backward_is_deterministic(globule20k):
    # sums in a fixed order (per source simplex, then per atom): bit-identical results, call after call
    c, r, gpu, ref, w, wt = globule20k
    dc0, dr0 = gpu.backward(wt)
    for _ in range(3):
        dc, dr = gpu.backward(wt)
        assert np.array_equal(dc.cpu().numpy(), dc0.cpu().numpy())
        assert np.array_equal(dr.cpu().numpy(), dr0.cpu().numpy())


def test_fp32_values_close_to_fp64(globule20k):
    # ac_eval_filtration_fp32: the same values in single precision (a measure, not part of the build)
    c, r, gpu, ref, w, wt = globule20k
    f32 = gpu.eval_filtration_fp32()
    rel = []
    for d in range(4):
        want = gpu.filtration_values(d).cpu().numpy()
        got = f32[d].cpu().numpy().astype(np.float64)
        assert got.shape == want.shape and np.all(np.isfinite(got))
        if d == 0:  # an unattached vertex is its own source: -r^2, exact in FP32
            own = ~gpu.attached(0).cpu().numpy().astype(bool)
            assert np.array_equal(got[own], want[own])
        nz = want != 0.0
        rel.append(np.abs(got[nz] - want[nz]) / np.abs(want[nz]))
    rel = np.concatenate(rel)
    assert np.median(rel) < 1e-5


def test_eval_at_inputs_reproduces_values(globule20k):
    import torch

    c, r, gpu, ref, w, wt = globule20k
    f = gpu.eval_filtration(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda())
    for d in range(4):
        want = gpu.filtration_values(d).cpu().numpy()
        got = f[d].cpu().numpy()
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9)


def test_autograd_function(globule20k):
    import torch

    import paper_1908_05944_gb300 as ac

    c, r, gpu, ref, w, wt = globule20k
    ct = torch.from_numpy(c).cuda().requires_grad_(True)
    rt = torch.from_numpy(r).cuda().requires_grad_(True)
    fs = ac.AlphaFiltration.apply(ct, rt, 0.0)
    loss = sum((f * wd).sum() for f, wd in zip(fs, wt))
    loss.backward()
    dc, dr = gpu.backward(wt)
    assert torch.allclose(ct.grad, dc, rtol=1e-12, atol=1e-12)
    assert torch.allclose(rt.grad, dr, rtol=1e-12, atol=1e-12)
