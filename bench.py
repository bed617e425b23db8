"""Benchmark: alpha complexes of synthetic atom sets on GB300 (atoms/s).

One step = one ac_build over the whole workload: quantisation, grid binning,
neighbour lists, the fused estimation + pruning pass (potential simplices and
AC2, Sections 4.3-4.4 / Steps 1-5 of arXiv 1908.05944), canonical lists and
Size filtration values. Inputs are resident in device memory when the timed
region starts; L2 is flushed (a 256 MB write) between timed steps.

`e2e` repeats the step through the public C ABI with host buffers: create from
pinned host arrays (host->device copy), build with every simplex list, its
filtration values and attached flags delivered to page-locked host memory
(opt.host_results), destroy.

With --impl reference the exact CPU oracle (oracle/) is timed instead, on a
bounded sub-ball of the same workload per step, on the host cores.

Multi-GPU: by default independent replicas (each rank builds its own copy;
value = atoms of all ranks / max-over-ranks time, weak scaling). With
--mode partitioned the ranks build the z-parts of one molecule from host
arrays (ac_build_part: each part with its halo, Section 4.6) and rank 0
gathers and merges the shares (ac_merge_parts); value = atoms of the molecule
/ max-over-ranks time of a step (strong scaling; host in, host out).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "alpha-complex atoms/s, plain vs filtered & batched, 100k/3M atoms; % roofline"
UNIT = "atoms/s"

# Algorithmic work of the per-atom pass, FP32 flops (an FMA counts 2), per unit:
# AC3 test of an edge / triangle / tetrahedron candidate (orthocentre solve) and
# one AC2 test of a (simplex, neighbour) pair: 3 FMA dot + 1 FMA + compare.
FLOPS_AC3 = {1: 20.0, 2: 60.0, 3: 120.0}
FLOPS_AC2 = 12.0
FP32_LANES_PER_SM = 128
SMS = 152
# GB300's FP64 rate is far below its FP32 rate: 1.25 TFLOP/s nominal at the
# 2,070 MHz maximum SM clock. The plain FP64 path is measured against it.
FP64_NOMINAL_TFLOPS = 1.25
MAX_SM_MHZ = 2070.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="globule100k_probe")
    p.add_argument("--precision", default="filtered", choices=["filtered", "plain_fp64"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the plain/shell side measurements")
    p.add_argument("--mode", default="replicas", choices=["replicas", "partitioned"],
                   help="replicas: every rank builds the whole workload (weak scaling); partitioned: the ranks "
                        "build the parts of one molecule and rank 0 merges them (strong scaling)")
    p.add_argument("--max-core-atoms", type=int, default=1 << 21, help="partitioned mode: atoms per slab of a part")
    return p.parse_args()


def local_device():
    """This rank's GPU: LOCAL_RANK, round-robin when ranks outnumber the GPUs (ranks then share one)."""
    import torch
    return int(os.environ.get("LOCAL_RANK", "0")) % max(1, torch.cuda.device_count())


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        # the only collectives are a barrier and a max of one number: NCCL with one GPU per rank,
        # gloo (host) when ranks share GPUs or for the reference arm
        backend = "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local_device())
            if world <= torch.cuda.device_count():
                backend = "nccl"
        dist.init_process_group(backend=backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons, sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self._t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(name):
    import synth
    return synth.workload(name)


def profiled_traffic(workload):
    """DRAM bytes per per-atom pass from the committed ncu summary, or None when
    the kernel source changed since that capture or the workload differs."""
    here = os.path.dirname(os.path.abspath(__file__))
    prof = os.path.join(here, "profiles", "k_local_globule100k.md")
    src = os.path.join(here, "paper_1908_05944_gb300", "csrc", "ac_local.cu")
    if workload != "globule100k_probe" or not (os.path.exists(prof) and os.path.exists(src)):
        return None
    fields = {}
    for ln in open(prof):
        if ":" in ln and ln.split(":", 1)[0] in ("traffic_bytes_per_pass", "source_sha256"):
            k, v = ln.split(":", 1)
            fields[k] = v.strip()
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    if fields.get("source_sha256") != sha or "traffic_bytes_per_pass" not in fields:
        return None
    return int(fields["traffic_bytes_per_pass"])


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


def algorithmic_flops(st):
    f = 0.0
    for d in (1, 2, 3):
        f += FLOPS_AC3[d] * st["ac3_tests"][d]
    f += FLOPS_AC2 * (sum(st["ac2_tests_tet"]) + sum(st["ac2_tests_tri"]) + st["ac2_tests_edge"])
    return f


def run_ours(args, rank, world):
    import torch

    import paper_1908_05944_gb300 as ac

    dev = local_device()
    torch.cuda.set_device(dev)
    c_np, r_np = workload(args.workload)
    n = len(r_np)
    prec = ac.AC_PRECISION_FILTERED if args.precision == "filtered" else ac.AC_PRECISION_PLAIN_FP64
    c = torch.from_numpy(c_np).cuda()
    r = torch.from_numpy(r_np).cuda()
    cx = ac.AlphaComplex(c, r, 0.0, ac.options(precision=prec))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        cx.build(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = []
    local_ms = []
    launches = 0
    flops = []
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            cx.build(stream)
            t1.record(stream)
            torch.cuda.synchronize()
            ms.append(t0.elapsed_time(t1))
            st = cx.stats()
            local_ms.append(st["ms_stage"][7])
            launches += st["kernel_launches"]
            flops.append(algorithmic_flops(st))
    torch.cuda.synchronize()
    barrier(world)
    total_ms = max_over_ranks(float(sum(ms)), world)
    st = cx.stats()
    counts = [cx.count(d) for d in range(4)]
    res = {
        "n_atoms": n,
        "ms_per_step": total_ms / args.steps,
        "value": n * world * args.steps / (total_ms / 1e3),
        "simplices_per_s": sum(counts) * world * args.steps / (total_ms / 1e3),
        "counts": counts,
        "stats": st,
        "local_ms": float(np.mean(local_ms)),
        "local_flops": float(np.mean(flops)),
        "launches": launches,
        "clocks": clk.summary(),
    }
    cx.close()
    return res


def time_builds(cx, steps, warmup, stream, flush):
    """Device time (ms) of each of `steps` builds after `warmup` untimed ones, L2 flushed in between."""
    import torch

    for _ in range(warmup):
        cx.build(stream)
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        cx.build(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        ms.append(t0.elapsed_time(t1))
    return ms


def measured_fma_peaks():
    """The device's FP32 and FP64 FMA throughput (TFLOP/s) from the library's probe (ac_fma_peak): independent
    FMA chains in registers over every SM, about 50 ms per timed launch, median of three."""
    import paper_1908_05944_gb300 as ac

    out = {}
    for name, fp64 in (("fp32_tflops", False), ("fp64_tflops", True)):
        out[name] = float(np.median([ac.fma_peak(fp64) for _ in range(3)])) / 1e12
    return out


def run_forms(args, fma=None):
    """Side measurements: plain FP64 vs filtered, the 3M shell, batched vs per-molecule launches."""
    import torch

    import paper_1908_05944_gb300 as ac
    import synth

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {}
    steps, warm = 3, 2
    for wl, prec in (("globule100k_probe", "plain_fp64"), ("shell3m_probe", "filtered"), ("shell3m_probe", "plain_fp64")):
        c_np, r_np = workload(wl)
        p = ac.AC_PRECISION_FILTERED if prec == "filtered" else ac.AC_PRECISION_PLAIN_FP64
        cx = ac.AlphaComplex(torch.from_numpy(c_np).cuda(), torch.from_numpy(r_np).cuda(), 0.0, ac.options(precision=p))
        ms = time_builds(cx, steps, warm, stream, flush)
        st = cx.stats()
        n = len(r_np)
        loc = st["ms_stage"][7]
        tf = algorithmic_flops(st) / (loc * 1e-3) / 1e12 if loc > 0 else 0.0
        out[f"{wl}/{prec}"] = {"atoms_per_s": n * steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps,
                               "simplices": st["simplices"], "local_kernel_ms": loc, "local_tflops": tf,
                               "local_frac_fp32_peak_2070mhz": tf / (SMS * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12)}
        if fma:
            out[f"{wl}/{prec}"]["local_frac_of_measured_fma"] = tf / fma["fp32_tflops" if prec == "filtered"
                                                                         else "fp64_tflops"]
        if prec == "plain_fp64":  # its bounding roofline: the FP64 pipe
            out[f"{wl}/{prec}"]["local_frac_fp64_nominal_2070mhz"] = tf / FP64_NOMINAL_TFLOPS
        if prec == "plain_fp64":
            # the filtered FP32 cascade against plain FP64 on the same input: lists and values
            fx = ac.AlphaComplex(torch.from_numpy(c_np).cuda(), torch.from_numpy(r_np).cuda(), 0.0).build(stream)
            same, worst = True, 0.0
            for d in range(4):
                same = same and torch.equal(fx.simplices(d), cx.simplices(d))
                same = same and torch.equal(fx.attached(d), cx.attached(d))
                f32, f64 = fx.filtration_values(d), cx.filtration_values(d)
                if f32.shape == f64.shape and f32.numel():
                    den = f64.abs().clamp_min(1e-300)
                    worst = max(worst, float(((f32 - f64).abs() / den).max()))
            out[f"{wl}/{prec}"]["filtered_vs_plain_fp64"] = {"lists_equal": bool(same), "f_max_rel_diff": worst}
            fx.close()
        cx.close()
        del cx
    # out-of-core build (Section 4.6): host arrays in, host lists out, z-slabs of at most max_core atoms
    # plus halo on the device at a time; against one whole-molecule build with the same host round trip
    c3, r3 = workload("shell3m_probe")
    reps = 3  # timed round trips of each kind after one untimed one (which also takes the page-locked blocks)
    whole_ms = []
    for rep in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        whole = ac.AlphaComplex(c3, r3, 0.0, ac.options(host_results=True)).build(stream)
        views = [whole.host_lists(d, copy=False) for d in range(4)]  # host lists made during the build
        if rep:
            whole_ms.append(1e3 * (time.perf_counter() - t0))
        if rep < reps:
            del views
            whole.close()
    host = [(t_.copy(), a_.copy(), f_.copy()) for t_, f_, a_ in views]  # kept past the context, untimed
    del views
    whole.close()
    del whole
    for max_core in (1_000_000, 250_000):
        runs = []
        for rep in range(reps + 1):
            t0 = time.perf_counter()
            ch = ac.ChunkedComplex(c3, r3, 0.0, max_core, stream=stream)
            wall = 1e3 * (time.perf_counter() - t0)
            if rep:
                runs.append((wall, ch.stats()))
            if rep < reps:
                ch.close()
        wall, st = sorted(runs, key=lambda x: x[0])[reps // 2]  # the median run
        equal = all(np.array_equal(ch.simplices(d), host[d][0]) and np.array_equal(ch.attached(d), host[d][1])
                    and np.array_equal(ch.filtration_values(d), host[d][2]) for d in range(4))
        out[f"shell3m_probe/chunked_{max_core}"] = {
            "atoms_per_s": len(r3) / (wall * 1e-3), "wall_ms": wall, "wall_ms_runs": [w for w, _ in runs],
            "n_chunks": st["n_chunks"], "subset_max": st["subset_max"],
            "halo_overhead": st["subset_total"] / len(r3) - 1.0,
            "ms_plan": st["ms_plan"], "ms_device": st["ms_device"], "ms_assemble": st["ms_assemble"],
            "equal_to_whole_build": bool(equal), "whole_build_host_round_trip_ms": float(np.median(whole_ms)),
            "whole_build_host_round_trip_ms_runs": whole_ms}
        ch.close()
        del ch
    del host
    # context for the paper's Table 1 row of its largest unpartitioned molecule (58,674 atoms, van der Waals
    # radii, alpha 0 and 1; 65 ms and 160 ms with memory transfers on a GTX 660 Ti): a synthetic globule of
    # the same size and radii, timed end to end (fresh context from host arrays, lists back in host memory)
    # and as a device-resident graph replay
    c58, r58 = synth.globule(7, 58674, probe=False)
    c58h, r58h = torch.from_numpy(c58).pin_memory(), torch.from_numpy(r58).pin_memory()
    for alpha in (0.0, 1.0):
        e2e = []
        for it in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ex = ac.AlphaComplex(c58h, r58h, alpha, ac.options(host_results=True)).build(stream)
            n_s = sum(ex.count(d) for d in range(4))
            ex.close()
            if it:
                e2e.append(time.perf_counter() - t0)
        gx = ac.AlphaComplex(torch.from_numpy(c58).cuda(), torch.from_numpy(r58).cuda(), alpha)
        ms = time_builds(gx, steps, warm, stream, flush)
        gx.close()
        out[f"globule58k_vdw/alpha{alpha:g}"] = {"simplices": int(n_s), "e2e_ms": 1e3 * float(np.median(e2e)),
                                               "device_ms": sum(ms) / steps,
                                               "paper_gtx660ti_ms_1AON": 65.2 if alpha == 0.0 else 159.9}
    # a point set unlike proteins: 200,000 particles (jittered lattice, radii log-uniform over a factor 8)
    cp, rp = synth.particles(13, 200000)
    px = ac.AlphaComplex(torch.from_numpy(cp).cuda(), torch.from_numpy(rp).cuda(), 0.0)
    ms = time_builds(px, steps, warm, stream, flush)
    pst = px.stats()
    out["particles200k"] = {"atoms_per_s": len(rp) * steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps,
                            "simplices": pst["simplices"], "max_degree": pst["max_degree"],
                            "neighbour_pairs_per_atom": pst["neighbour_pairs"] / len(rp)}
    px.close()
    # the same cloud with radii over a factor of 16: dozens of atoms per thousand have 513..1,024
    # neighbours (32-word rows, working sets in global memory)
    cw, rw = synth.particles(15, 200000, r_hi=4.0)
    wx = ac.AlphaComplex(torch.from_numpy(cw).cuda(), torch.from_numpy(rw).cuda(), 0.0)
    ms = time_builds(wx, steps, warm, stream, flush)
    wst = wx.stats()
    out["particles200k_wide"] = {"atoms_per_s": len(rw) * steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps,
                                 "simplices": wst["simplices"], "max_degree": wst["max_degree"],
                                 "neighbour_pairs_per_atom": wst["neighbour_pairs"] / len(rw),
                                 "local_kernel_ms": wst["ms_stage"][7]}
    wx.close()
    # batch: one context over all molecules vs one context per molecule
    sizes = synth.batch_sizes(4, 1024)
    mols = [synth.globule(1000 + m, int(n), probe=True) for m, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum([len(r) for _, r in mols])])
    c_all = torch.from_numpy(np.concatenate([m[0] for m in mols])).cuda()
    r_all = torch.from_numpy(np.concatenate([m[1] for m in mols])).cuda()
    n_all = int(offsets[-1])
    bx = ac.AlphaComplex(c_all, r_all, 0.0, offsets=offsets)
    tuned = bx.autotune(stream)
    ms = time_builds(bx, steps, warm, stream, flush)
    batched = n_all * steps / (sum(ms) / 1e3)
    replayed = bx.stats()["replayed"]
    bx.close()
    del bx
    # the comparison: one context per molecule, every build synchronised (no graph)
    singles = [ac.AlphaComplex(c_all[offsets[m]:offsets[m + 1]], r_all[offsets[m]:offsets[m + 1]], 0.0,
                               ac.options(no_graph=True)) for m in range(len(mols))]
    for cx in singles:
        cx.build(stream)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for cx in singles:
        cx.build(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    per_mol = n_all / (t0.elapsed_time(t1) / 1e3)
    for cx in singles:
        cx.close()
    out["batch1024_probe"] = {"n_atoms": n_all, "batched_atoms_per_s": batched, "batched_ms": sum(ms) / steps,
                              "batched_graph_replay": bool(replayed), "autotuned": tuned,
                              "per_molecule_atoms_per_s": per_mol}
    # alpha sweep (the filtration restricted): one build at alpha = 2 A^2, then the complexes at 21 alphas in
    # [0, 2] by exact thresholds on Size, against 21 separate builds
    cg, rg = workload("globule100k_probe")
    tc, tr = torch.from_numpy(cg).cuda(), torch.from_numpy(rg).cuda()
    alphas2 = [0.1 * k for k in range(21)]
    sx = ac.AlphaComplex(tc, tr, 2.0).build(stream)
    sx.build(stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sx.build(stream)
    sizes = [[sx.subcomplex_mask(d, a2, -1, stream)[1] for d in range(4)] for a2 in alphas2]
    torch.cuda.synchronize()
    sweep_ms = (time.perf_counter() - t0) * 1e3
    sx.close()
    t0 = time.perf_counter()
    for a2 in alphas2:
        bx2 = ac.AlphaComplex(tc, tr, a2).build(stream)
        bx2.close()
    torch.cuda.synchronize()
    builds_ms = (time.perf_counter() - t0) * 1e3
    out["globule100k_probe/alpha_sweep"] = {"alphas": len(alphas2), "sweep_ms": sweep_ms, "separate_builds_ms": builds_ms,
                                           "simplices_at_0_and_2": [sizes[0], sizes[-1]]}
    # backward (row a14) on the 20k globule: dL/dcentres, dL/dradii for random weights on every simplex
    c20, r20 = workload("globule20k_probe")
    gx = ac.AlphaComplex(torch.from_numpy(c20).cuda(), torch.from_numpy(r20).cuda(), 0.0).build(stream)
    rng = np.random.default_rng(synth.LOSS_WEIGHT_SEED)
    dldf = [torch.from_numpy(rng.standard_normal(gx.count(d))).cuda() for d in range(4)]
    for _ in range(2):
        gx.backward(dldf, stream)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(5):
        gx.backward(dldf, stream)
    t1.record(stream)
    torch.cuda.synchronize()
    bms = t0.elapsed_time(t1) / 5
    # the filtration values in FP32 arithmetic against the build's (exact rationals rounded to FP64)
    cg, rg = workload("globule100k_probe")
    fx = ac.AlphaComplex(torch.from_numpy(cg).cuda(), torch.from_numpy(rg).cuda(), 0.0).build(stream)
    f32 = fx.eval_filtration_fp32(stream)
    rel, zeros = [], 0
    for d in range(4):
        want = fx.filtration_values(d).cpu().numpy()
        got = f32[d].cpu().numpy().astype(np.float64)
        nz = want != 0.0
        zeros += int((~nz).sum())
        rel.append(np.abs(got[nz] - want[nz]) / np.abs(want[nz]))
    fx.close()
    rel = np.concatenate(rel)
    out["globule100k_probe/fp32_filtration_error"] = {
        "rel_err_max": float(rel.max()), "rel_err_p50": float(np.median(rel)), "rel_err_p99": float(np.percentile(rel, 99)),
        "values": int(rel.size), "exact_zeros_skipped": zeros,
        "what": "each simplex's value (its source's OrthoSize) in FP32 arithmetic from the quantised inputs, "
                "against the build's FP64 values (exact rationals rounded once)"}
    out["globule20k_probe/backward"] = {"ms_per_call": bms, "atoms_per_s": len(r20) / (bms / 1e3),
                                        "simplices": [gx.count(d) for d in range(4)]}
    gx.close()
    return out


def run_e2e(args, rank, world, steps):
    """Whole public-API round trip with host buffers: a fresh context from page-locked host arrays
    (H2D inside), one build that also delivers every list (rows, filtration values, attached flags)
    to host memory (opt.host_results: each list is copied as soon as it is final, overlapping the
    rest of the build), and the context's destruction."""
    import torch

    import paper_1908_05944_gb300 as ac

    c_np, r_np = workload(args.workload)
    n = len(r_np)
    c_h = torch.from_numpy(c_np).pin_memory()
    r_h = torch.from_numpy(r_np).pin_memory()
    prec = ac.AC_PRECISION_FILTERED if args.precision == "filtered" else ac.AC_PRECISION_PLAIN_FP64
    h2d = c_np.nbytes + r_np.nbytes
    times = []
    d2h = 0
    for it in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cx = ac.AlphaComplex(c_h, r_h, 0.0, ac.options(precision=prec, host_results=True))
        cx.build()
        d2h = 0
        for d in range(4):
            t, f, a = cx.host_lists(d, copy=False)  # page-locked host memory, filled by the build
            d2h += t.nbytes + f.nbytes + a.nbytes
        cx.close()
        if it > 0:  # the first round trip warms the allocators
            times.append(time.perf_counter() - t0)
    t = max_over_ranks(float(sum(times)), world)
    return {"value": n * world * steps / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def cpu_baseline(args):
    """The oracle, as it stands, on the whole workload (all host cores), and on the whole 2,000-atom
    and 20,000-atom configurations; the GPU lists compared with it."""
    import oracle

    c, r = workload(args.workload)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    res = oracle.alpha_complex(c, r, 0.0, threads=threads, candidates=False)
    dt = time.perf_counter() - t0
    out = {"value": len(r) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"the whole {args.workload} ({len(r)} atoms), 1 run, {dt:.2f} s",
           "simplices": int(sum(res.counts())), "parity": parity_on(c, r, res)}
    for wl in ("globule2k_vdw", "globule20k_probe"):
        c0, r0 = workload(wl)
        t0 = time.perf_counter()
        oracle.alpha_complex(c0, r0, 0.0, threads=threads, candidates=False)
        dt = time.perf_counter() - t0
        out[wl] = {"atoms_per_s": len(r0) / dt, "atoms": len(r0), "seconds": dt}
    return out


def parity_on(c, r, ref):
    """The GPU complex of the same atoms against the oracle's: lists (bit-exact) and Size values."""
    import torch

    import paper_1908_05944_gb300 as ac

    out = {}
    for name, prec in (("filtered", ac.AC_PRECISION_FILTERED), ("plain_fp64", ac.AC_PRECISION_PLAIN_FP64)):
        cx = ac.AlphaComplex(torch.from_numpy(c).cuda(), torch.from_numpy(r).cuda(), 0.0, ac.options(precision=prec))
        cx.build()
        same, rel = True, []
        for d in range(4):
            got = cx.simplices(d).cpu().numpy()
            same &= got.shape == ref.simplices[d].shape and bool(np.array_equal(got, ref.simplices[d]))
            same &= bool(np.array_equal(cx.attached(d).cpu().numpy().astype(bool), ref.attached[d]))
            if same:
                f, g = cx.filtration_values(d).cpu().numpy(), ref.f[d]
                nz = g != 0
                same &= bool(np.array_equal(f[~nz], g[~nz]))
                rel.append(np.abs(f[nz] - g[nz]) / np.abs(g[nz]))
        cx.close()
        rel = np.concatenate(rel) if rel else np.zeros(1)
        out[name] = {"lists_equal": same, "f_rel_err_max": float(rel.max()), "f_rel_err_p50": float(np.median(rel)),
                     "f_rel_err_p99": float(np.percentile(rel, 99))}
    return out


def sub_ball(c, r, k):
    centre = np.median(c, axis=0)
    d = np.linalg.norm(c - centre, axis=1)
    idx = np.sort(np.argsort(d)[:k])
    return c[idx], r[idx]


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle

    c, r = workload(args.workload)
    # about 0.7 s of oracle work per 20,000-atom step on 16 cores: smaller samples when many steps
    # are asked for, so that the whole run stays within a few minutes
    sample_atoms = int(min(20000, max(2000, 20000 * 100 // max(1, args.steps + args.warmup))))
    sc, sr = sub_ball(c, r, sample_atoms)
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.alpha_complex(sc, sr, 0.0, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.alpha_complex(sc, sr, 0.0, threads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = len(sr) * args.steps / tot
    sample = f"{len(sr)}-atom sub-ball of {args.workload} per step"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64/int128 (exact)",
        "data": "synthetic", "config": {"workload": args.workload, "alpha": 0.0, "sample_atoms": len(sr)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_partitioned(args, rank, world):
    """One molecule over the ranks: part build (host arrays in, host lists out), gather and merge on rank 0."""
    import torch
    import torch.distributed as dist

    import paper_1908_05944_gb300 as ac

    dev = local_device()
    torch.cuda.set_device(dev)
    c, r = workload(args.workload)
    n = len(r)
    group = dist.new_group(backend="gloo") if world > 1 else None  # the shares cross in host memory
    stream = torch.cuda.current_stream()

    def step():
        part = ac.ChunkedComplex.part(c, r, 0.0, world, rank, args.max_core_atoms, stream=stream)
        share = part.share()
        part.close()
        if world == 1:
            return ac.merge_parts(n, [share])
        got = [None] * world if rank == 0 else None
        dist.gather_object(share, got, dst=0, group=group)
        return ac.merge_parts(n, got) if rank == 0 else None

    for _ in range(args.warmup):
        m = step()
        if m is not None:
            m.close()
    times = []
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            barrier(world)
            t0 = time.perf_counter()
            m = step()
            barrier(world)
            times.append(time.perf_counter() - t0)
            counts = [m.count(d) for d in range(4)] if m is not None else None
            if m is not None:
                m.close()
    total = max_over_ranks(float(sum(times)), world)
    if rank != 0:
        return None
    value = n * args.steps / total
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32 filter, f64/int128 exact fallback", "data": "synthetic",
        "config": {"workload": args.workload, "n_atoms": n, "alpha": 0.0, "parallelism": f"parts x{world}",
                   "max_core_atoms": args.max_core_atoms, "l2": "inputs and lists in host memory (larger than L2)"},
        "clocks": clk.summary(), "simplices": counts,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(c.nbytes + r.nbytes),
                "d2h_bytes_per_step": None},
    }


def main():
    args = parse()
    rank, world = dist_init(args)
    if args.impl == "ours" and args.mode == "partitioned":
        import importlib
        if rank == 0:
            importlib.import_module("paper_1908_05944_gb300.build").build()
        barrier(world)
        line = run_partitioned(args, rank, world)
        if rank == 0:
            print(json.dumps(line))
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if rank == 0:
            print(json.dumps(line))
        return
    import torch  # noqa: F401

    import importlib
    if rank == 0:  # one process compiles (if the library is stale); the others wait for it
        importlib.import_module("paper_1908_05944_gb300.build").build()
    barrier(world)
    res = run_ours(args, rank, world)
    peaks = measured_peaks()
    clocks = res["clocks"]
    sm_mhz = clocks.get("sm_mhz") or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 2070.0
    if args.precision == "filtered":
        peak_tflops = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        basis = f"FP32 FMA: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz (derived; sampled SM clock)"
    else:
        peak_tflops = FP64_NOMINAL_TFLOPS * sm_mhz / MAX_SM_MHZ
        basis = (f"FP64: nominal {FP64_NOMINAL_TFLOPS} TFLOP/s at {MAX_SM_MHZ:.0f} MHz, scaled to the sampled "
                 f"{sm_mhz:.0f} MHz")
    achieved = res["local_flops"] / (res["local_ms"] * 1e-3) / 1e12 if res["local_ms"] > 0 else 0.0
    fma = measured_fma_peaks()  # after the timed steps
    measured = fma["fp32_tflops" if args.precision == "filtered" else "fp64_tflops"]
    line = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 filter, f64/int128 exact fallback" if args.precision == "filtered"
        else "f64 filter, int128 exact fallback",
        "data": "synthetic",
        "config": {"workload": args.workload, "n_atoms": res["n_atoms"], "alpha": 0.0,
                   "precision": args.precision, "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{world}"},
        "simplices_per_s": res["simplices_per_s"],
        "simplices": res["counts"],
        "clocks": clocks,
        "gpu_launches": res["launches"],
        "roofline": {"bound": "alu", "kernel": "k_local (fused estimation + pruning)", "achieved": achieved,
                     "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops if peak_tflops else None,
                     "traffic": profiled_traffic(args.workload) if args.precision == "filtered" else None,
                     "traffic_unit": "bytes per pass (ncu dram read + write, both launches)",
                     "peak_basis": basis,
                     "peak_measured_fma": measured,
                     "frac_of_measured_fma": achieved / measured if measured else None},
        "fma_peaks_measured": fma,
        "stage_ms": res["stats"]["ms_stage"],
        "predicates": {"ac2_tet": res["stats"]["ac2_tests_tet"], "ac2_tri": res["stats"]["ac2_tests_tri"],
                       "ac2_edge": res["stats"]["ac2_tests_edge"], "ac3": res["stats"]["ac3_tests"]},
    }
    if not args.no_e2e:
        line["e2e"] = run_e2e(args, rank, world, max(2, min(args.steps, 5)))
    if rank == 0 and world == 1 and not args.no_forms:
        line["forms"] = run_forms(args, fma)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
