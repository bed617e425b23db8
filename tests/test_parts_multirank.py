"""One molecule over two processes (Section 4.6: parts of the grid, each with its
border), the host side on CPU: world size 2 over gloo.

The device build of a part (ac_build_part) needs a GPU and is tested in
test_gpu_parts.py. Here each rank takes its share from the oracle's complex
of the whole molecule by the same rule ac_build_part follows (the rows whose
first vertex has its quantised z in the rank's range of ac_part_plan); the
shares cross between the processes with torch.distributed.gather_object, as
distributed_complex sends them, and ac_merge_parts places them. The merged
lists must equal the whole complex row for row. Also: the cut of ac_part_plan
(ranges in order, atoms split about evenly), and the merge's refusals
(overlapping shares, a share out of order, a vertex out of range).
"""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _molecule():
    return synth.globule(31, 1500, probe=True)


def _share(ref, z, lo, hi):
    """The rows of the oracle's complex whose first vertex v has lo <= Z_v < hi."""
    out = []
    for d in range(4):
        t = ref.simplices[d]
        keep = (z[t[:, 0]] >= lo) & (z[t[:, 0]] < hi) if len(t) else np.zeros(0, bool)
        out.append((t[keep], ref.f[d][keep], ref.attached[d][keep].astype(np.uint8)))
    return out


def _z_quanta(c):
    return np.rint(c[:, 2] * 1024.0).astype(np.int64)  # round half to even, as the library quantises


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    import paper_1908_05944_gb300 as ac

    dist.init_process_group("gloo", rank=rank, world_size=world)
    c, r = _molecule()
    thr, _ = ac.part_plan(c, r, 0.0, world)
    ref = oracle.alpha_complex(c, r, 0.0, threads=2)
    share = _share(ref, _z_quanta(c), thr[rank], thr[rank + 1])
    got = [None] * world if rank == 0 else None
    dist.gather_object(share, got, dst=0)
    if rank == 0:
        merged = ac.merge_parts(len(r), got)
        ok = all(np.array_equal(merged.simplices(d), ref.simplices[d]) and
                 np.array_equal(merged.filtration_values(d), ref.f[d]) and
                 np.array_equal(merged.attached(d).astype(bool), ref.attached[d]) for d in range(4))
        sizes = [len(s[1][0]) for s in got]
        with open(os.path.join(out_dir, "result.txt"), "w") as fh:
            fh.write(f"{int(ok)} {sizes[0]} {sizes[1]}")
    dist.destroy_process_group()


def test_two_ranks_gather_and_merge(tmp_path):
    import torch.multiprocessing as mp

    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    ok, e0, e1 = (int(x) for x in (tmp_path / "result.txt").read_text().split())
    assert ok == 1
    assert e0 > 0 and e1 > 0  # both ranks held part of the edges


def test_part_plan_splits_evenly():
    import paper_1908_05944_gb300 as ac

    c, r = _molecule()
    z = _z_quanta(c)
    for k in (1, 2, 3, 7):
        thr, reach = ac.part_plan(c, r, 0.0, k)
        assert len(thr) == k + 1 and thr[0] == z.min() and thr[-1] == z.max() + 1
        assert np.all(np.diff(thr) >= 0)
        counts = np.histogram(z, bins=thr)[0] if k > 1 else np.array([len(z)])
        assert counts.sum() == len(z)
        assert counts.max() <= len(z) / k + 64  # cuts at histogram bins of one quantum here
    assert reach == 2 * int(np.ceil(np.sqrt((np.rint(r * 1024) ** 2).max())))


def test_merge_of_one_share_and_of_shares_in_any_order():
    import paper_1908_05944_gb300 as ac

    c, r = _molecule()
    ref = oracle.alpha_complex(c, r, 0.0)
    z = _z_quanta(c)
    thr, _ = ac.part_plan(c, r, 0.0, 3)
    shares = [_share(ref, z, thr[p], thr[p + 1]) for p in range(3)]
    for order in ([0, 1, 2], [2, 0, 1]):
        m = ac.merge_parts(len(r), [shares[p] for p in order])
        for d in range(4):
            assert np.array_equal(m.simplices(d), ref.simplices[d])
            assert np.array_equal(m.filtration_values(d), ref.f[d])
    whole = ac.merge_parts(len(r), [_share(ref, z, z.min(), z.max() + 1)])
    assert np.array_equal(whole.simplices(3), ref.simplices[3])
    empty = ac.merge_parts(0, [])
    assert all(empty.count(d) == 0 for d in range(4))


def test_merge_refuses_bad_shares():
    import paper_1908_05944_gb300 as ac

    c, r = _molecule()
    ref = oracle.alpha_complex(c, r, 0.0)
    z = _z_quanta(c)
    full = _share(ref, z, z.min(), z.max() + 1)
    with pytest.raises(ac.AlphacError) as e:  # two shares with the same first vertices
        ac.merge_parts(len(r), [full, full])
    assert e.value.code == ac.AC_ERR_INVALID_ARG
    rev = [(t[::-1].copy(), f[::-1].copy(), a[::-1].copy()) for t, f, a in full]
    with pytest.raises(ac.AlphacError):  # rows not in first-vertex order
        ac.merge_parts(len(r), [rev])
    with pytest.raises(ac.AlphacError):  # a vertex beyond n
        ac.merge_parts(len(r) - 1, [full])
