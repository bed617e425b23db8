"""Parity at the benchmark sizes, in the launch configuration bench.py times.

Every configuration is compared whole with the oracle, list by list:
* 100,000-atom globule (probe radii), both predicate modes;
* 3,000,000-atom capsid-like shell: one oracle run over all of it;
* 1,024 molecules of uneven sizes (10.7 M atoms) in one batched context,
  autotuned and replayed as a graph: every molecule against its own oracle
  run (the runs spread over the host cores), and the per-molecule row ranges
  partition every list.
Plus properties that hold at any size (closure under faces, monotone Size) on
the shell.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_complex, host_lists, lists_differ, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("mode", [0, 1], ids=["filtered", "plain_fp64"])
def test_globule100k_whole(mode):
    c, r = synth.workload("globule100k_probe")
    ref = oracle.alpha_complex(c, r, 0.0)
    gpu = run_gpu(c, r, 0.0, precision=mode)
    assert_same_complex(gpu, ref)
    st = gpu.stats()
    assert st["candidates"][1:] == [int(x) for x in ref.candidate_counts()[1:]]


@pytest.fixture(scope="module")
def shell():
    c, r = synth.workload("shell3m_probe")
    gpu = run_gpu(c, r, 0.0)
    gpu.build()  # the replayed build, as timed by the bench
    assert gpu.stats()["replayed"] == 1
    out = {"c": c, "r": r, "L": host_lists(gpu), "stats": gpu.stats()}
    out["S"] = [x[0] for x in out["L"]]
    out["F"] = [x[2] for x in out["L"]]
    gpu.close()
    return out


def test_shell3m_whole(shell):
    ref = oracle.alpha_complex(shell["c"], shell["r"], 0.0, candidates=False)
    err = lists_differ(shell["L"], ref)
    assert err is None, err


def test_shell3m_closure_and_monotone_size(shell):
    S, F = shell["S"], shell["F"]
    rng = np.random.default_rng(7)
    for d in range(1, 4):
        lower = S[d - 1]
        keys = lower.astype(np.int64)
        # lexicographic search in the sorted lower list
        view = np.ascontiguousarray(keys).view([("", np.int64)] * d).ravel()
        rows = rng.choice(len(S[d]), min(200000, len(S[d])), replace=False)
        for drop in range(d + 1):
            faces = np.delete(S[d][rows], drop, axis=1).astype(np.int64)
            fv = np.ascontiguousarray(faces).view([("", np.int64)] * d).ravel()
            pos = np.searchsorted(view, fv)
            assert np.all(pos < len(view))
            assert np.array_equal(keys[pos], faces), f"dim {d}: a face is missing"
            assert np.all(F[d - 1][pos] <= F[d][rows]), f"dim {d}: Size not monotone"
    st = shell["stats"]
    n = len(shell["r"])
    per_atom = sum(st["simplices"]) / n
    assert 5 < per_atom < 40


def test_batch1024_every_molecule(tmp_path):
    from concurrent.futures import ThreadPoolExecutor

    import torch

    import paper_1908_05944_gb300 as ac

    mols = synth.batch()
    offsets = np.concatenate([[0], np.cumsum([len(r) for _, r in mols])])
    c_all = torch.from_numpy(np.concatenate([m[0] for m in mols])).cuda()
    r_all = torch.from_numpy(np.concatenate([m[1] for m in mols])).cuda()
    bx = ac.AlphaComplex(c_all, r_all, 0.0, offsets=offsets)
    tuned = bx.autotune()
    bx.build()
    bx.build()  # the replayed build, as timed by the bench
    assert bx.stats()["replayed"] == 1
    sizes = np.diff(offsets)
    # every row belongs to exactly one molecule, whose atoms it indexes
    st = bx.stats()
    lists = [host_lists(bx, m) for m in range(len(mols))]
    for d in range(4):
        assert sum(len(lists[m][d][0]) for m in range(len(mols))) == st["simplices"][d]
        for m in range(len(mols)):
            t = lists[m][d][0]
            if len(t):
                assert int(t.min()) >= 0 and int(t.max()) < sizes[m]
    bx.close()

    workers = max(1, min(8, (os.cpu_count() or 2) // 2))

    def check(m):
        cm, rm = mols[m]
        ref = oracle.alpha_complex(cm, rm, 0.0, threads=2, candidates=False)
        err = lists_differ(lists[m], ref)
        return None if err is None else f"molecule {m} ({sizes[m]} atoms): {err}"

    with ThreadPoolExecutor(workers) as ex:  # ctypes releases the GIL: oracle runs overlap
        errors = [e for e in ex.map(check, range(len(mols))) if e]
    if errors:
        # which path differs: a synchronised build (no graph) of the same batch, same plan
        sx = ac.AlphaComplex(c_all, r_all, 0.0, ac.options(no_graph=True, **tuned), offsets=offsets).build()
        bad = [int(e.split()[1]) for e in errors]
        sync = [host_lists(sx, m) for m in range(len(mols))]
        sx.close()
        sync_ok = [lists_differ(sync[m], oracle.alpha_complex(*mols[m], 0.0, candidates=False)) is None for m in bad[:5]]
        report = {"plan": tuned, "n_bad": len(bad), "sync_matches_oracle": sync_ok, "dims": {}}
        for d in range(4):
            cr = np.array([len(lists[m][d][0]) for m in range(len(mols))])
            cs = np.array([len(sync[m][d][0]) for m in range(len(mols))])
            rows = [m for m in range(len(mols)) if cr[m] == cs[m] and not np.array_equal(lists[m][d][0], sync[m][d][0])]
            vals = [m for m in range(len(mols)) if cr[m] == cs[m] and np.array_equal(lists[m][d][0], sync[m][d][0])
                    and not np.array_equal(lists[m][d][2], sync[m][d][2])]
            report["dims"][d] = {"count_mismatch": int((cr != cs).sum()), "total_r": int(cr.sum()),
                                 "total_s": int(cs.sum()), "rows_mismatch": len(rows), "vals_mismatch": len(vals),
                                 "nan": int(sum(np.isnan(lists[m][d][2]).sum() for m in range(len(mols)))),
                                 "first": [(int(m), int(cr[m]), int(cs[m])) for m in np.nonzero(cr != cs)[0][:5]]}
        import json

        path = tmp_path / "batch_fail.json"
        path.write_text(json.dumps(report, indent=1))
        errors.append(f"plan {tuned}; {len(bad)} molecules differ; a synchronised build matches the oracle: "
                      f"{sync_ok}; per-dimension report in {path}")
    assert not errors, errors[:5] + errors[-1:]
