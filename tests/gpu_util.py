"""Helpers shared by the GPU tests: run the library and the oracle on the same input and compare."""
import numpy as np

F_RTOL = 1e-12  # filtration values: relative tolerance; exact zeros must match exactly


def run_gpu(centres, radii, alpha=0.0, **opt):
    import torch

    import paper_1908_05944_gb300 as ac

    c = torch.as_tensor(np.asarray(centres, dtype=np.float64)).cuda()
    r = torch.as_tensor(np.asarray(radii, dtype=np.float64)).cuda()
    return ac.AlphaComplex(c, r, alpha, ac.options(**opt) if opt else None).build()


def assert_same_complex(gpu, ref, check_values=True, mol=-1):
    for d in range(4):
        got = gpu.simplices(d, mol).cpu().numpy()
        want = ref.simplices[d]
        assert got.shape == want.shape, f"dim {d}: {got.shape[0]} simplices on the GPU, {want.shape[0]} in the oracle"
        if not np.array_equal(got, want):
            bad = np.nonzero(np.any(got != want, axis=1))[0][:5]
            raise AssertionError(f"dim {d}: first differing rows {bad}: gpu {got[bad]} oracle {want[bad]}")
        att = gpu.attached(d, mol).cpu().numpy().astype(bool)
        assert np.array_equal(att, ref.attached[d]), f"dim {d}: attached flags differ"
        if check_values:
            f = gpu.filtration_values(d, mol).cpu().numpy()
            assert_values(f, ref.f[d], f"dim {d}")


def assert_values(got, want, what=""):
    zero = want == 0.0
    assert np.array_equal(got[zero], want[zero]), f"{what}: exact zeros differ"
    nz = ~zero
    rel = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
    if rel.size:
        worst = int(np.argmax(rel))
        assert rel[worst] <= F_RTOL, f"{what}: relative error {rel[worst]:.3e} at {worst}"


def host_lists(gpu, mol=-1):
    """Rows, attached flags and filtration values of every dimension, copied to host memory."""
    return [(gpu.simplices(d, mol, copy=False).cpu().numpy(), gpu.attached(d, mol, copy=False).cpu().numpy().astype(bool),
             gpu.filtration_values(d, mol, copy=False).cpu().numpy()) for d in range(4)]


def lists_differ(lists, ref):
    """None if host lists (from host_lists) equal the oracle's complex, else what differs first."""
    for d, (rows, att, f) in enumerate(lists):
        want = ref.simplices[d]
        if rows.shape != want.shape:
            return f"dim {d}: {rows.shape[0]} simplices on the GPU, {want.shape[0]} in the oracle"
        if not np.array_equal(rows, want):
            bad = np.nonzero(np.any(rows != want, axis=1))[0][:3]
            return f"dim {d}: rows {bad} differ: gpu {rows[bad].tolist()} oracle {want[bad].tolist()}"
        if not np.array_equal(att, ref.attached[d]):
            return f"dim {d}: attached flags differ"
        try:
            assert_values(f, ref.f[d], f"dim {d}")
        except AssertionError as e:
            return str(e)
    return None
