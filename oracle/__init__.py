"""Exact CPU oracle for the alpha complex of weighted points (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may
import this package. The CUDA library never does, and the two share no code:
this wrapper loads ``alpha_oracle.c`` (compiled with gcc into ``_build/``),
which follows the paper's Steps 1-5 (Section 3.1) in exact integer arithmetic.

Returned simplices are tuples of INPUT indices, each tuple ascending, each list
sorted lexicographically. Filtration values are Size (Section 2.3) in A^2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alpha_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", -1: "invalid argument", -2: "degenerate (coincident centres)", -3: "out of range",
          -5: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, 'unknown')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle into an in-tree shared library (gcc; no GPU needed)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _open(path):
    """A ctypes handle on an oracle library at ``path`` with its signatures declared."""
    lib = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.oracle_run.restype = ctypes.c_int
    lib.oracle_run.argtypes = [vp, vp, i64, dbl, i32, i32, ctypes.POINTER(vp)]
    lib.oracle_count.restype = i64
    lib.oracle_count.argtypes = [vp, i32, i32]
    lib.oracle_copy_simplices.restype = None
    lib.oracle_copy_simplices.argtypes = [vp, i32, i32, vp]
    lib.oracle_copy_values.restype = None
    lib.oracle_copy_values.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    lib.oracle_gradient.restype = ctypes.c_int
    lib.oracle_gradient.argtypes = [vp, vp, vp, vp]
    lib.oracle_free.restype = None
    lib.oracle_free.argtypes = [vp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _open(_LIB_PATH)
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class AlphaComplex:
    """Result of one oracle run. ``simplices[d]`` is an int32 array (count, d+1).

    ``candidates[d]`` holds Sigma_ortho^d unless the run was made with
    candidates=False (then it is empty: the lists stay in the C result, which
    saves host memory at millions of atoms).
    """

    def __init__(self, handle, n: int, lib, with_candidates: bool = True):
        self._h = handle
        self.n = n
        self._lib = lib
        self.simplices = []
        self.candidates = []
        self.f = []
        self.orthosize = []
        self.attached = []
        self.src_dim = []
        self.src_idx = []
        for d in range(4):
            m = lib.oracle_count(handle, 0, d)
            s = np.zeros((m, d + 1), dtype=np.int32)
            if m:
                lib.oracle_copy_simplices(handle, 0, d, s.ctypes.data)
            self.simplices.append(s)
            c = lib.oracle_count(handle, 1, d) if with_candidates else 0
            cs = np.zeros((c, d + 1), dtype=np.int32)
            if c:
                lib.oracle_copy_simplices(handle, 1, d, cs.ctypes.data)
            self.candidates.append(cs)
            f = np.zeros(m, dtype=np.float64)
            o = np.zeros(m, dtype=np.float64)
            a = np.zeros(m, dtype=np.uint8)
            sd = np.zeros(m, dtype=np.int32)
            si = np.zeros(m, dtype=np.int64)
            if m:
                lib.oracle_copy_values(handle, d, f.ctypes.data, o.ctypes.data, a.ctypes.data, sd.ctypes.data,
                                       si.ctypes.data)
            self.f.append(f)
            self.orthosize.append(o)
            self.attached.append(a.astype(bool))
            self.src_dim.append(sd)
            self.src_idx.append(si)

    def counts(self):
        return [len(s) for s in self.simplices]

    def candidate_counts(self):
        return [len(s) for s in self.candidates]

    def gradient(self, dldf):
        """Closed-form dL/dcentres (n,3) and dL/dradii (n,) for L = sum_d dldf[d] . f[d]."""
        lib = self._lib
        arrs = []
        ptrs = (ctypes.c_void_p * 4)()
        for d in range(4):
            w = None if dldf[d] is None else np.ascontiguousarray(dldf[d], dtype=np.float64)
            arrs.append(w)
            ptrs[d] = None if w is None else w.ctypes.data
        dc = np.zeros((self.n, 3), dtype=np.float64)
        dr = np.zeros(self.n, dtype=np.float64)
        rc = lib.oracle_gradient(self._h, ctypes.cast(ptrs, ctypes.c_void_p), dc.ctypes.data, dr.ctypes.data)
        if rc != 0:
            raise OracleError(rc)
        return dc, dr

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and getattr(self, "_lib", None) is not None:
            self._lib.oracle_free(h)


def alpha_complex(centres, radii, alpha: float = 0.0, alpha_inf: bool = False, threads: int | None = None,
                  lib_path: str | None = None, candidates: bool = True):
    """Run the exact oracle. centres (n,3) and radii (n,) in A; alpha in A^2.

    lib_path selects another build of the oracle source (the mutation test uses it).
    candidates=False leaves the Sigma_ortho lists out of the returned object.
    """
    lib = _load() if lib_path is None else _open(lib_path)
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
    r = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    if len(c) != len(r):
        raise ValueError("centres and radii differ in length")
    h = ctypes.c_void_p()
    rc = lib.oracle_run(c.ctypes.data, r.ctypes.data, len(r), float(alpha), 1 if alpha_inf else 0,
                        threads or default_threads(), ctypes.byref(h))
    if rc != 0:
        raise OracleError(rc)
    return AlphaComplex(h, len(r), lib, with_candidates=candidates)
