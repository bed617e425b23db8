"""Reader for the hand-derived fixtures in tests/golden/ (atoms, alpha, expected complex)."""
from __future__ import annotations

import glob
import os
from fractions import Fraction

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_fixture(path):
    atoms, alpha, expect = [], None, {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "atom":
                atoms.append(tuple(Fraction(t) for t in tok[1:5]))
            elif tok[0] == "alpha":
                alpha = None if tok[1] == "inf" else Fraction(tok[1])
            elif tok[0] == "simplex":
                verts = tuple(int(t) for t in tok[1:] if "=" not in t)
                kv = dict(t.split("=") for t in tok[1:] if "=" in t)
                expect[verts] = (Fraction(kv["f"]), kv["attached"] == "1")
    return atoms, alpha, expect


def fixtures():
    return sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))
