"""bench.py's own multi-rank paths under torchrun, two ranks on one GPU.

With more ranks than GPUs the ranks share a GPU (round-robin) and the
bench's two collectives (a barrier, the max of the elapsed time) run over
gloo; the ranks' kernels never wait on one another.
* replicas: every rank builds the whole workload; one JSON line from rank 0.
* partitioned: the ranks build the two parts of one molecule, rank 0 merges;
  the merged complex has the whole build's simplex counts.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

import synth
from gpu_util import run_gpu

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(*extra):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--gpus", "2", "--workload", "globule20k_probe", *extra]
    res = subprocess.run(cmd, cwd=ROOT, env=dict(os.environ, OMP_NUM_THREADS="2"), capture_output=True, text=True,
                         timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    return json.loads(lines[0])


def test_replicas_two_ranks():
    line = _torchrun("--steps", "2", "--warmup", "1", "--no-e2e", "--no-forms", "--no-cpu-baseline")
    assert line["n_gpus"] == 2 and line["scaling"] == "weak" and line["value"] > 0
    assert line["config"]["parallelism"] == "replicas x2"
    c, r = synth.workload("globule20k_probe")
    g = run_gpu(c, r, 0.0)
    assert line["simplices"] == [g.count(d) for d in range(4)]


def test_partitioned_two_ranks():
    line = _torchrun("--mode", "partitioned", "--steps", "1", "--warmup", "0", "--max-core-atoms", "6000")
    assert line["n_gpus"] == 2 and line["scaling"] == "strong" and line["value"] > 0
    assert line["config"]["parallelism"] == "parts x2"
    c, r = synth.workload("globule20k_probe")
    g = run_gpu(c, r, 0.0)
    assert line["simplices"] == [g.count(d) for d in range(4)]
