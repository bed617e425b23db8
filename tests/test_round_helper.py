"""The int128 -> double rounding of the exact filtration values (csrc/ac_round.h),
compiled for the host with g++ and checked against Python, whose int -> float
conversion is correctly rounded (nearest, ties to even): random magnitudes up
to 2^126, values exactly halfway between two doubles (both tie directions),
just below and above a halfway point, powers of two, carries that round up
to the next power of two, and the 2^-20 scaling.
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
#include <string.h>
#include "ac_round.h"
int main() {
    char buf[128];
    int e2;
    while (scanf("%127s %d", buf, &e2) == 2) {
        const char* p = buf;
        bool neg = *p == '-';
        if (neg) p++;
        unsigned __int128 u = 0;
        for (; *p; p++) u = u * 10 + (unsigned)(*p - '0');
        __int128 x = neg ? -(__int128)u : (__int128)u;
        double d = ac::i128_to_double_rn(x, e2);
        unsigned long long b;
        memcpy(&b, &d, sizeof b);
        printf("%016llx\n", b);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("round")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    return str(exe)


def _run(exe, cases):
    inp = "".join(f"{x} {e}\n" for x, e in cases)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    return [int(h, 16) for h in out]


def _bits(v):
    import struct

    return struct.unpack("<Q", struct.pack("<d", v))[0]


def _want(x, e2):
    # exact scaling by a power of two after the one rounding (results stay normal)
    return _bits(float(x) * 2.0**e2)


def test_matches_correct_rounding(harness):
    rng = random.Random(7)
    cases = []
    for _ in range(20000):
        nb = rng.randint(1, 126)
        x = rng.getrandbits(nb) | (1 << (nb - 1))
        cases.append((x if rng.random() < 0.5 else -x, rng.choice((0, -20))))
    for k in range(54, 127):
        base = rng.getrandbits(53) | (1 << 52)
        sh = k - 53
        half = 1 << (sh - 1)
        for m in (base, base | 1, (1 << 53) - 1):
            for r in (half, half - 1, half + 1, 0, (1 << sh) - 1):
                cases.append(((m << sh) + r, 0))
                cases.append((-((m << sh) + r), -20))
    for k in range(0, 127):
        cases.append((1 << k, 0))
        cases.append((-(1 << k), -20))
        cases.append(((1 << k) - 1 if k else 1, 0))
    got = _run(harness, cases)
    assert len(got) == len(cases)
    bad = [(x, e, hex(g), hex(_want(x, e))) for (x, e), g in zip(cases, got) if g != _want(x, e)]
    assert not bad, bad[:5]


def test_zero(harness):
    assert _run(harness, [(0, 0), (0, -20)]) == [0, 0]
