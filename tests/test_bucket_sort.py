"""The one-thread sort of large canonicalisation buckets (csrc/ac_bucket.h),
compiled for the host with g++ and checked against a plain Python sort: for
K = 2, 3 (w a flag, OR-ed over equal tuples) and K = 4 (w part of the key),
buckets of 0 to 5,000 tuples with many repeats, already sorted, reversed and
all-equal inputs, and a bucket in the middle of a larger array (the items
around it must stay untouched). A third check counts the key comparisons on
buckets of 10^5 tuples: at most 3 k log2 k, so the sort stays O(k log k) (an
insertion sort, quadratic, took minutes on the GPU for such buckets).
"""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1908_05944_gb300", "csrc")

HARNESS = r"""
#include <stdio.h>
#include <vector>
#include "ac_bucket.h"
struct Tup { int x, y, z, w; };
int main() {
    int K;
    long long n, a, b;
    while (scanf("%d %lld %lld %lld", &K, &n, &a, &b) == 4) {
        std::vector<Tup> T(n);
        for (auto& t : T)
            if (scanf("%d %d %d %d", &t.x, &t.y, &t.z, &t.w) != 4) return 1;
        long long u = K == 2 ? ac::sort_unique_bucket<2>(T.data(), a, b)
                    : K == 3 ? ac::sort_unique_bucket<3>(T.data(), a, b)
                             : ac::sort_unique_bucket<4>(T.data(), a, b);
        printf("%lld\n", u);
        for (const auto& t : T) printf("%d %d %d %d\n", t.x, t.y, t.z, t.w);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("bucket")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    return str(exe)


def _run(exe, cases):
    inp = []
    for K, T, a, b in cases:
        inp.append(f"{K} {len(T)} {a} {b}\n")
        inp.extend(f"{x} {y} {z} {w}\n" for x, y, z, w in T)
    out = subprocess.run([exe], input="".join(inp), capture_output=True, text=True, check=True).stdout.split("\n")
    res, k = [], 0
    for K, T, a, b in cases:
        u = int(out[k])
        rows = [tuple(int(v) for v in out[k + 1 + i].split()) for i in range(len(T))]
        res.append((u, rows))
        k += 1 + len(T)
    return res


def _want(K, T, a, b):
    """The sorted distinct tuples of T[a:b] (for K < 4, w OR-ed over equal tuples)."""
    seg = T[a:b]
    if K == 4:
        uniq = sorted(set(seg), key=lambda t: (t[1], t[2], t[3]))
    else:
        flags = {}
        for x, y, z, w in seg:
            flags[(x, y, z)] = flags.get((x, y, z), 0) | w
        uniq = [(x, y, z, f) for (x, y, z), f in sorted(flags.items(), key=lambda kv: (kv[0][1], kv[0][2]))]
    return uniq


def _bucket(rng, K, n, span):
    x = 17
    out = []
    for _ in range(n):
        y = rng.randrange(span)
        z = rng.randrange(span) if K >= 3 else -1
        w = rng.randrange(span) if K == 4 else rng.randrange(2)
        out.append((x, y, z, w))
    return out


def test_sort_unique_matches_python(harness):
    rng = random.Random(3)
    cases = []
    for K in (2, 3, 4):
        for n in (0, 1, 2, 3, 7, 257, 1000, 5000):
            for span in (3, 40, 100000):
                cases.append((K, _bucket(rng, K, n, span), 0, n))
        base = _bucket(rng, K, 2000, 30)
        cases.append((K, sorted(base, key=lambda t: (t[1], t[2], t[3])), 0, 2000))
        cases.append((K, sorted(base, key=lambda t: (t[1], t[2], t[3]), reverse=True), 0, 2000))
        cases.append((K, [(17, 5, 6 if K >= 3 else -1, 1 if K == 4 else i % 2) for i in range(600)], 0, 600))
    got = _run(harness, cases)
    for (K, T, a, b), (u, rows) in zip(cases, got):
        want = _want(K, T, a, b)
        assert u == len(want), (K, len(T))
        assert rows[a:a + u] == want, (K, len(T))


def test_bucket_inside_a_larger_array(harness):
    rng = random.Random(4)
    for K in (2, 3, 4):
        T = _bucket(rng, K, 3000, 50)
        a, b = 700, 2600
        (u, rows), = _run(harness, [(K, T, a, b)])
        assert rows[:a] == T[:a] and rows[b:] == T[b:], "items outside the bucket changed"
        assert u == len(_want(K, T, a, b))
        assert rows[a:a + u] == _want(K, T, a, b)


COUNTING = r"""
#include <stdio.h>
#include <vector>
#include "ac_bucket.h"
static long long g_cmp = 0;
struct CInt {  // an int whose comparisons are counted
    int v;
    bool operator<(const CInt& o) const { ++g_cmp; return v < o.v; }
    bool operator!=(const CInt& o) const { ++g_cmp; return v != o.v; }
    bool operator==(const CInt& o) const { ++g_cmp; return v == o.v; }
    CInt& operator|=(const CInt& o) { v |= o.v; return *this; }
};
struct Tup { CInt x, y, z, w; };
int main() {
    long long n;
    int kind;
    while (scanf("%lld %d", &n, &kind) == 2) {
        std::vector<Tup> T(n);
        unsigned s = 12345u;
        for (long long i = 0; i < n; i++) {
            s = s * 1664525u + 1013904223u;
            int y = kind == 0 ? (int)(s >> 8) % 1000000 : kind == 1 ? (int)i : (int)(n - i);
            T[i] = Tup{{17}, {y}, {(int)(s >> 20) & 7}, {(int)(s >> 3) & 1}};
        }
        g_cmp = 0;
        long long u = ac::sort_unique_bucket<4>(T.data(), 0, n);
        bool sorted = true;
        for (long long i = 1; i < u; i++) {
            const Tup &a = T[i - 1], &b = T[i];
            if (a.y.v > b.y.v || (a.y.v == b.y.v && (a.z.v > b.z.v || (a.z.v == b.z.v && a.w.v >= b.w.v))))
                sorted = false;
        }
        printf("%lld %lld %d\n", g_cmp, u, sorted ? 1 : 0);
    }
    return 0;
}
"""


def test_comparisons_are_n_log_n(tmp_path):
    import math

    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "c.cpp"
    src.write_text(COUNTING)
    exe = tmp_path / "c"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    n = 100000
    inp = "".join(f"{n} {kind}\n" for kind in (0, 1, 2))  # random, ascending, descending
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for line in out[:3]:
        cmp, u, ok = (int(v) for v in line.split())
        assert ok == 1 and 0 < u <= n
        # each key comparison is up to 3 field comparisons (y, z, w); the de-duplication adds 3 per tuple
        assert cmp <= 3 * (3 * n * math.log2(n)) + 3 * n, (cmp, n)
