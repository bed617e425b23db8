"""ac_backward_noalloc: the backward without device allocation, through the C ABI.

Some callers cannot allocate device memory at all (a training step whose
memory belongs to another allocator, a service with a fixed device budget);
this entry point serves them by keeping the backward's small pointer table in
a static device array. Its gradients must equal ac_backward's (to rounding:
its kernel adds with atomics, ac_backward in a fixed order), call after call,
also when calls alternate between contexts, and a call must not take memory
from the device's memory pool. This file is collected last so that a failure
here comes after every other test has run; it also passes on its own in a
fresh process.
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
        # FP64 atomics accumulate in no fixed order: agree to rounding
        _close(dc, dc_ref)
        _close(dr, dr_ref)


def _second():
    import torch

    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(78, 2500, probe=True)
    cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0).build()
    counts = [cx.count(d) for d in range(4)]
    w = synth.normal(92, sum(counts))
    ws, k = [], 0
    for d in range(4):
        ws.append(torch.from_numpy(w[k:k + counts[d]].copy()).cuda())
        k += counts[d]
    return cx, ws


def _close(got, want):
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_noalloc_backward_alternating_contexts(built):
    # the shared table is rewritten for each call's context: alternate two contexts of different sizes
    ac, cx, ws = built
    cy, wy = _second()
    L = ac.lib()
    _, dcx, drx = _call(L.ac_backward, cx, ws, cx.n)
    _, dcy, dry = _call(L.ac_backward, cy, wy, cy.n)
    for _ in range(2):
        for ctx, w, dc_ref, dr_ref in ((cx, ws, dcx, drx), (cy, wy, dcy, dry)):
            rc, dc, dr = _call(L.ac_backward_noalloc, ctx, w, ctx.n)
            assert rc == ac.AC_OK, ac.lib().ac_last_error_detail()
            _close(dc, dc_ref)
            _close(dr, dr_ref)
    cy.close()


def _pool_used_bytes():
    """Bytes in use in the current device's default stream-ordered memory pool (the pool the library allocates from)."""
    import glob

    names = ["libcudart.so"] + sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*"))
    rt = None
    for name in names:
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    if rt is None:
        pytest.skip("libcudart not found")
    dev = ctypes.c_int()
    assert rt.cudaGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used = ctypes.c_uint64()
    cudaMemPoolAttrUsedMemCurrent = 7
    assert rt.cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, ctypes.byref(used)) == 0
    return used.value


def test_noalloc_backward_takes_no_pool_memory(built):
    # on a fresh context that never ran ac_backward: the pool's bytes in use do not change across the call
    import torch

    ac, _, _ = built
    cz, wz = _second()
    torch.cuda.synchronize()
    before = _pool_used_bytes()
    rc, dc, _ = _call(ac.lib().ac_backward_noalloc, cz, wz, cz.n)
    torch.cuda.synchronize()
    assert rc == ac.AC_OK
    assert np.all(np.isfinite(dc))
    assert _pool_used_bytes() == before
    cz.close()


def test_noalloc_backward_refuses_unbuilt_context(built):
    import torch

    ac, cx, ws = built
    fresh = ac.AlphaComplex(torch.zeros((1, 3), dtype=torch.float64).cuda(), torch.ones(1, dtype=torch.float64).cuda())
    empty = [torch.zeros(0, dtype=torch.float64, device="cuda")] * 4
    rc, _, _ = _call(ac.lib().ac_backward_noalloc, fresh, empty, 1)
    assert rc == ac.AC_ERR_STATE
