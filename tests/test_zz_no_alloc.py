"""ac_backward_noalloc: the backward without device allocation, through the C ABI.

Some callers cannot allocate device memory at all (a training step whose
memory belongs to another allocator, a service with a fixed device budget);
this entry point serves them by keeping the backward's small pointer table in
a static device array. Its gradients must equal ac_backward's, call after
call. This file is collected last so that a failure here comes after every
other test has run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import importlib

    importlib.import_module("paper_1908_05944_gb300.build").build()
    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(77, 6000, probe=True)
    cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0).build()
    counts = [cx.count(d) for d in range(4)]
    w = synth.normal(91, sum(counts))
    ws, k = [], 0
    for d in range(4):
        ws.append(torch.from_numpy(w[k:k + counts[d]].copy()).cuda())
        k += counts[d]
    return ac, cx, ws


def _call(entry, cx, ws, n):
    import torch

    ptrs = (ctypes.c_void_p * 4)(*[wd.data_ptr() if wd.numel() else None for wd in ws])
    dc = torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda")
    dr = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = entry(cx._h, ctypes.cast(ptrs, ctypes.c_void_p), dc.data_ptr(), dr.data_ptr(), stream)
    return rc, dc.cpu().numpy(), dr.cpu().numpy()


def test_noalloc_backward_matches_backward_twice(built):
    ac, cx, ws = built
    L = ac.lib()
    rc, dc_ref, dr_ref = _call(L.ac_backward, cx, ws, cx.n)
    assert rc == ac.AC_OK
    for _ in range(2):
        rc, dc, dr = _call(L.ac_backward_noalloc, cx, ws, cx.n)
        assert rc == ac.AC_OK, ac.lib().ac_last_error_detail()
        assert np.all(np.isfinite(dc)) and np.all(np.isfinite(dr))
        # FP64 atomics accumulate in a different order: agree to rounding
        np.testing.assert_allclose(dc, dc_ref, rtol=1e-12, atol=1e-12 * np.abs(dc_ref).max())
        np.testing.assert_allclose(dr, dr_ref, rtol=1e-12, atol=1e-12 * np.abs(dr_ref).max())


def test_noalloc_backward_refuses_unbuilt_context(built):
    import torch

    ac, cx, ws = built
    fresh = ac.AlphaComplex(torch.zeros((1, 3), dtype=torch.float64).cuda(), torch.ones(1, dtype=torch.float64).cuda())
    empty = [torch.zeros(0, dtype=torch.float64, device="cuda")] * 4
    rc, _, _ = _call(ac.lib().ac_backward_noalloc, fresh, empty, 1)
    assert rc == ac.AC_ERR_STATE
