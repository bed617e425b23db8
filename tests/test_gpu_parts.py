"""One molecule built in parts on the GPU (Section 4.6: parts of the grid, each
with its border) and merged: ac_build_part + ac_merge_parts, through the C ABI.

* In one process: the parts of a 1, 2, 3 or 5-way cut (with slabs inside a
  part when max_core_atoms is small), merged, equal the whole build and the
  oracle, row for row, with flags and values.
* Two processes on one GPU over gloo (distributed_complex): each rank builds
  its part on cuda:0, rank 0 gathers and merges. The ranks' kernels never
  wait on one another (independent builds; the exchange is on the host).
"""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_complex, host_lists, lists_differ, run_gpu

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _host_of(merged):
    return [(merged.simplices(d), merged.attached(d).astype(bool), merged.filtration_values(d)) for d in range(4)]


@pytest.mark.parametrize("parts,max_core", [(1, 1 << 21), (2, 1 << 21), (3, 700), (5, 1 << 21)])
def test_parts_merge_to_whole(parts, max_core):
    import paper_1908_05944_gb300 as ac

    c, r = synth.globule(41, 6000, probe=True)
    ref = oracle.alpha_complex(c, r, 0.0)
    whole = run_gpu(c, r, 0.0)
    assert_same_complex(whole, ref)
    shares = []
    for p in range(parts):
        part = ac.ChunkedComplex.part(c, r, 0.0, parts, p, max_core)
        shares.append(part.share())
        part.close()
    merged = ac.merge_parts(len(r), shares)
    err = lists_differ(_host_of(merged), ref)
    assert err is None, err
    # the same rows as the device lists of the whole build
    for d in range(4):
        assert np.array_equal(merged.simplices(d), whole.simplices(d).cpu().numpy())


def test_parts_alpha_and_ties():
    import paper_1908_05944_gb300 as ac

    # equal-z lattice layers (cuts between and within ties) at alpha > 0
    rng = np.random.default_rng(5)
    g = np.stack(np.meshgrid(np.arange(9), np.arange(9), np.arange(9), indexing="ij"), -1).reshape(-1, 3) * 1.5
    c = g[rng.permutation(len(g))]
    r = np.full(len(c), 1.25)
    ref = oracle.alpha_complex(c, r, 0.5)
    shares = []
    for p in range(4):
        part = ac.ChunkedComplex.part(c, r, 0.5, 4, p, 1 << 21)
        shares.append(part.share())
        part.close()
    err = lists_differ(_host_of(ac.merge_parts(len(r), shares, 0.5)), ref)
    assert err is None, err


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist

    import paper_1908_05944_gb300 as ac

    torch.cuda.set_device(0)  # one GPU: both ranks build their parts on it
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c, r = synth.globule(43, 8000, probe=True)
    merged = ac.distributed_complex(c, r, 0.0, max_core_atoms=3000)
    if rank == 0:
        ref = oracle.alpha_complex(c, r, 0.0)
        err = lists_differ(_host_of(merged), ref)
        with open(os.path.join(out_dir, "result.txt"), "w") as fh:
            fh.write("ok" if err is None else err)
    else:
        assert merged is None
    dist.destroy_process_group()


def test_two_ranks_on_one_gpu(tmp_path):
    import torch.multiprocessing as mp

    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    assert (tmp_path / "result.txt").read_text() == "ok"
