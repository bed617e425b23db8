"""Seeded synthetic weighted-atom inputs (no alpha-complex arithmetic here).

The generator recipe is documented in ``synth/synth.c``. It stands in for the
biomolecules of the paper's experiments (Section 5): centres by random
sequential addition at 0.05 atoms/A^3 with a 1.3 A minimum separation, element
radii C/N/O/S (optionally grown by a 1.4 A solvent probe), alpha = 0.

Every coordinate and radius it returns is an exact multiple of 1/1024 A, so
the library's quantisation (round half even of 1024 x) reproduces the integer
values it drew.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

DENSITY = 0.05  # atoms per A^3


def build(force: bool = False) -> str:
    """Compile synth.c into an in-tree shared library (gcc, no GPU needed)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.synth_atoms.restype = ctypes.c_int
            lib.synth_atoms.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_batch_sizes.restype = None
            lib.synth_batch_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_void_p]
            lib.synth_normal.restype = None
            lib.synth_normal.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            lib.synth_raw.restype = None
            lib.synth_raw.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            _lib = lib
    return _lib


def ball_radius(n: int, density: float = DENSITY) -> float:
    """Radius (A) of the ball that holds n atoms at the given density."""
    return (3.0 * n / (4.0 * math.pi * density)) ** (1.0 / 3.0)


def atoms_int(seed: int, n: int, r_out: float, r_in: float = -1.0, probe: bool = True):
    """Quantised atoms: (xyz int32 n x 3, radius int32 n, element uint8 n), 1/1024 A units."""
    lib = _load()
    xyz = np.zeros((n, 3), dtype=np.int32)
    rad = np.zeros(n, dtype=np.int32)
    el = np.zeros(n, dtype=np.uint8)
    if n > 0:
        rc = lib.synth_atoms(seed, n, r_in, r_out, 1 if probe else 0, xyz.ctypes.data, rad.ctypes.data,
                             el.ctypes.data)
        if rc != 0:
            raise RuntimeError(f"synth_atoms failed with code {rc}")
    return xyz, rad, el


def atoms(seed: int, n: int, r_out: float, r_in: float = -1.0, probe: bool = True):
    """Atoms in A: (centres float64 n x 3, radii float64 n), exact multiples of 1/1024."""
    xyz, rad, _ = atoms_int(seed, n, r_out, r_in, probe)
    return xyz.astype(np.float64) / 1024.0, rad.astype(np.float64) / 1024.0


def globule(seed: int, n: int, probe: bool = True):
    """A protein-like globule: n atoms in the ball of radius ball_radius(n)."""
    return atoms(seed, n, ball_radius(n), -1.0, probe)


def batch_sizes(seed: int, n_mol: int, lo: float = 500.0, hi: float = 50000.0) -> np.ndarray:
    lib = _load()
    out = np.zeros(n_mol, dtype=np.int64)
    lib.synth_batch_sizes(seed, n_mol, lo, hi, out.ctypes.data)
    return out


def normal(seed: int, n: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(n, dtype=np.float64)
    if n > 0:
        lib.synth_normal(seed, n, out.ctypes.data)
    return out


def raw(seed: int, k: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(k, dtype=np.uint64)
    lib.synth_raw(seed, k, out.ctypes.data)
    return out


def particles(seed: int, n: int, spacing: float = 1.0, r_lo: float = 0.25, r_hi: float = 2.0):
    """A particle set unlike a protein (an SPH-like cloud): n points on a jittered cubic lattice of the
    given spacing (each coordinate moved by up to 0.4 spacing, so no two coincide), radii log-uniform in
    [r_lo, r_hi] (a ratio of 8 by default, against about 1.2 for atoms). Centres and radii are exact
    multiples of 1/1024 (units as for atoms)."""
    u = (raw(seed, 4 * n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 if n else np.zeros(0)
    u = u.reshape(n, 4) if n else np.zeros((0, 4))
    m = max(1, int(math.ceil(n ** (1.0 / 3.0) - 1e-9)))
    k = np.arange(n)
    lattice = np.stack([k % m, (k // m) % m, k // (m * m)], 1).astype(np.float64)
    xyz = (lattice + (u[:, :3] - 0.5) * 0.8) * spacing
    r = r_lo * (r_hi / r_lo) ** u[:, 3]
    return np.round(xyz * 1024.0) / 1024.0, np.round(r * 1024.0) / 1024.0


# The five workloads (sizes, regions, seeds), named by what they are.
WORKLOADS = {
    "globule2k_vdw": dict(seed=1, n=2000, probe=False),
    "globule100k_probe": dict(seed=2, n=100000, probe=True),
    "shell3m_probe": dict(seed=3, n=3000000, probe=True, r_in=320.0, r_out=361.0),
    "batch1024_probe": dict(seed=4, n_mol=1024, probe=True),
    "globule20k_probe": dict(seed=5, n=20000, probe=True),
}
LOSS_WEIGHT_SEED = 6


def workload(name: str):
    """(centres, radii) for a single-molecule workload, in A."""
    w = WORKLOADS[name]
    if "n_mol" in w:
        raise ValueError("use batch() for the batched workload")
    if "r_in" in w:
        return atoms(w["seed"], w["n"], w["r_out"], w["r_in"], w["probe"])
    return globule(w["seed"], w["n"], w["probe"])


def batch(n_mol: int | None = None, seed: int = 4, probe: bool = True):
    """The batched workload: molecule m uses seed 1000+m and the log-uniform size draw."""
    sizes = batch_sizes(seed, 1024)
    if n_mol is not None:
        sizes = sizes[:n_mol]
    mols = []
    for m, n in enumerate(sizes):
        mols.append(globule(1000 + m, int(n), probe))
    return mols
