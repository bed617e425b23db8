"""Host-side pieces of the benchmark (no GPU): the algorithmic work count behind
the roofline, and the rule that the DRAM traffic of the per-atom kernel is
reported only while its source is the one the ncu capture was taken on."""
import hashlib
import importlib.util
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join("paper_1908_05944_gb300", "csrc", "ac_local.cu")
PROFILE = os.path.join("profiles", "k_local_globule100k.md")


def _load_bench(root=ROOT):
    spec = importlib.util.spec_from_file_location("bench_host_mod", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_flops_counts_every_test_once():
    bench = _load_bench()
    st = {"ac3_tests": [0, 7, 5, 3], "ac2_tests_tet": [11, 2, 1], "ac2_tests_tri": [13, 1, 0], "ac2_tests_edge": 17}
    # per unit: edge AC3 20, triangle AC3 60, tetrahedron AC3 120, one AC2 test 12 (all levels of the cascade)
    want = 20 * 7 + 60 * 5 + 120 * 3 + 12 * (11 + 2 + 1 + 13 + 1 + 0 + 17)
    assert bench.algorithmic_flops(st) == want
    # vertex AC3 is a comparison, not arithmetic: it does not count
    st["ac3_tests"][0] = 10**6
    assert bench.algorithmic_flops(st) == want


def test_fp32_peak_basis():
    bench = _load_bench()
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA at 2070 MHz
    assert abs(bench.SMS * bench.FP32_LANES_PER_SM * 2 * 2070e6 / 1e12 - 80.54784) < 1e-9


def _profile_fields():
    fields = {}
    for ln in open(os.path.join(ROOT, PROFILE)):
        if ":" in ln:
            k, v = ln.split(":", 1)
            fields[k.strip()] = v.strip()
    return fields


def test_profiled_traffic_follows_the_source_hash(tmp_path):
    fields = _profile_fields()
    assert int(fields["traffic_bytes_per_pass"]) > 0
    assert len(fields["source_sha256"]) == 64
    # a copy of the three files the rule reads, with the hash made to match
    for rel in ("bench.py", PROFILE, SRC):
        os.makedirs(os.path.dirname(os.path.join(tmp_path, rel)) or str(tmp_path), exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), os.path.join(tmp_path, rel))
    src = os.path.join(tmp_path, SRC)
    prof = os.path.join(tmp_path, PROFILE)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    text = open(prof).read().replace(fields["source_sha256"], sha)
    open(prof, "w").write(text)
    bench = _load_bench(str(tmp_path))
    assert bench.profiled_traffic("globule100k_probe") == int(fields["traffic_bytes_per_pass"])
    assert bench.profiled_traffic("shell3m_probe") is None  # captured on another workload
    # any change to the kernel source voids the figure
    with open(src, "a") as f:
        f.write("\n// edited\n")
    assert bench.profiled_traffic("globule100k_probe") is None
