"""Python binding of alphac (include/alphac.h): alpha complexes of weighted atoms on one GPU.

The binding only marshals arguments to the C ABI of ``_build/libalphac.so``;
every step of the computation runs in the library's CUDA kernels. There is no
CPU fallback: if the library is missing or cannot be loaded, calls raise.

Method: Masood, Ray, Natarajan, "Parallel Computation of Alpha Complexes for
Biomolecules" (arXiv 1908.05944): potential simplices bottom-up (Section 4.3),
pruning by the empty-orthosphere test AC2 (Section 4.4), Size filtration values
(Section 2.3).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libalphac.so")

AC_OK = 0
AC_ERR_INVALID_ARG = -1
AC_ERR_DEGENERATE = -2
AC_ERR_RANGE = -3
AC_ERR_CAPACITY = -4
AC_ERR_OOM = -5
AC_ERR_CUDA = -6
AC_ERR_TIMEOUT = -7
AC_ERR_STATE = -8
AC_PRECISION_FILTERED = 0
AC_PRECISION_PLAIN_FP64 = 1
AC_FILTRATION_SIZE = 0
AC_FILTRATION_ORTHOSIZE = 1

# every symbol include/alphac.h declares
EXPORTS = ["ac_create", "ac_create_batch", "ac_build", "ac_get_simplices", "ac_filtration_values", "ac_attached_flags",
           "ac_get_candidates", "ac_eval_filtration", "ac_eval_filtration_fp32", "ac_backward", "ac_backward_noalloc", "ac_autotune",
           "ac_subcomplex", "ac_get_simplices_host", "ac_chunk_plan", "ac_build_chunked", "ac_part_plan", "ac_build_part",
           "ac_merge_parts", "ac_chunked_simplices", "ac_chunked_info",
           "ac_chunked_free", "ac_get_stats", "ac_get_sizes", "ac_destroy", "ac_error_string", "ac_last_error_detail",
           "ac_fma_peak"]


class ac_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("filtration", ctypes.c_int32), ("cell_factor", ctypes.c_double),
                ("block_warps", ctypes.c_int32), ("keep_candidates", ctypes.c_int32),
                ("no_graph", ctypes.c_int32), ("host_results", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


class ac_stats(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("candidates", ctypes.c_int64 * 4), ("simplices", ctypes.c_int64 * 4),
                ("neighbour_pairs", ctypes.c_int64), ("max_degree", ctypes.c_int32), ("grid_dims", ctypes.c_int32 * 3),
                ("ac2_tests_tet", ctypes.c_int64 * 3), ("ac2_tests_tri", ctypes.c_int64 * 3),
                ("ac2_tests_edge", ctypes.c_int64), ("ac3_tests", ctypes.c_int64 * 4), ("ac3_exact", ctypes.c_int64),
                ("ms_total", ctypes.c_double),
                ("ms_stage", ctypes.c_double * 8), ("kernel_launches", ctypes.c_int64),
                ("replayed", ctypes.c_int32), ("host_syncs", ctypes.c_int32), ("escalated", ctypes.c_int64)]

    def to_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class ac_chunked_stats(ctypes.Structure):
    _fields_ = [("n_chunks", ctypes.c_int64), ("reach", ctypes.c_int64), ("core_max", ctypes.c_int64),
                ("subset_max", ctypes.c_int64), ("subset_total", ctypes.c_int64), ("ms_plan", ctypes.c_double),
                ("ms_device", ctypes.c_double), ("ms_assemble", ctypes.c_double)]


class AlphacError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        msg = f"{where}: {error_string(code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)
        self.code = code


_lib = None
_lock = threading.Lock()


def _declare(lib):
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    lib.ac_create.argtypes = [vp, vp, i64, dbl, P(ac_options), P(vp)]
    lib.ac_create_batch.argtypes = [vp, vp, vp, i64, dbl, P(ac_options), P(vp)]
    lib.ac_build.argtypes = [vp, vp]
    lib.ac_fma_peak.argtypes = [i32, i32, vp, P(dbl), P(ctypes.c_float)]
    lib.ac_get_simplices.argtypes = [vp, i32, i64, P(vp), P(i64)]
    lib.ac_filtration_values.argtypes = [vp, i32, i64, P(vp), P(i64)]
    lib.ac_attached_flags.argtypes = [vp, i32, i64, P(vp), P(i64)]
    lib.ac_get_candidates.argtypes = [vp, i32, P(vp), P(i64)]
    lib.ac_eval_filtration.argtypes = [vp, vp, vp, vp, vp]
    lib.ac_eval_filtration_fp32.argtypes = [vp, vp, vp]
    lib.ac_backward.argtypes = [vp, vp, vp, vp, vp]
    lib.ac_backward_noalloc.argtypes = [vp, vp, vp, vp, vp]
    lib.ac_autotune.argtypes = [vp, vp, P(ac_options)]
    lib.ac_subcomplex.argtypes = [vp, i32, i64, dbl, vp, P(i64), vp]
    lib.ac_get_simplices_host.argtypes = [vp, i32, i64, P(vp), P(vp), P(vp), P(i64)]
    lib.ac_chunk_plan.argtypes = [vp, vp, i64, dbl, i64, vp, i64, P(i64), P(i64)]
    lib.ac_build_chunked.argtypes = [vp, vp, i64, dbl, P(ac_options), i64, vp, P(vp)]
    lib.ac_part_plan.argtypes = [vp, vp, i64, dbl, i64, vp, P(i64)]
    lib.ac_build_part.argtypes = [vp, vp, i64, dbl, P(ac_options), i64, i64, i64, vp, P(vp)]
    lib.ac_merge_parts.argtypes = [i64, i64, vp, vp, vp, vp, P(vp)]
    lib.ac_chunked_simplices.argtypes = [vp, i32, P(vp), P(vp), P(vp), P(i64)]
    lib.ac_chunked_info.argtypes = [vp, P(ac_chunked_stats)]
    lib.ac_chunked_free.argtypes = [vp]
    lib.ac_chunked_free.restype = None
    lib.ac_get_stats.argtypes = [vp, P(ac_stats)]
    lib.ac_get_sizes.argtypes = [vp, P(i64), P(i64)]
    lib.ac_destroy.argtypes = [vp]
    lib.ac_destroy.restype = None
    lib.ac_error_string.argtypes = [i32]
    lib.ac_error_string.restype = ctypes.c_char_p
    lib.ac_last_error_detail.argtypes = []
    lib.ac_last_error_detail.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("ac_destroy", "ac_chunked_free", "ac_error_string", "ac_last_error_detail"):
            getattr(lib, name).restype = ctypes.c_int


def lib():
    """The loaded libalphac.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"alphac library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
            handle = ctypes.CDLL(LIB_PATH)
            _declare(handle)
            _lib = handle
    return _lib


def error_string(code: int) -> str:
    return lib().ac_error_string(code).decode()


def _check(rc: int, where: str):
    if rc != AC_OK:
        raise AlphacError(rc, where, lib().ac_last_error_detail().decode())


def _ptr(a):
    """Data pointer of a torch tensor or numpy array (contiguous, correct dtype expected)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _as_f64(a):
    if hasattr(a, "data_ptr"):
        import torch
        return a.detach().to(torch.float64).contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class _DeviceArray:
    """Non-owning __cuda_array_interface__ view of device memory owned by a context."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}


def options(precision=AC_PRECISION_FILTERED, filtration=AC_FILTRATION_SIZE, cell_factor=0.0, block_warps=0,
            keep_candidates=False, no_graph=False, host_results=False) -> ac_options:
    o = ac_options()
    o.host_results = 1 if host_results else 0
    o.precision = precision
    o.filtration = filtration
    o.cell_factor = cell_factor
    o.block_warps = block_warps
    o.keep_candidates = 1 if keep_candidates else 0
    o.no_graph = 1 if no_graph else 0
    return o


class AlphaComplex:
    """One ac_ctx: created from centres (n,3) and radii (n,) in A and alpha in A^2.

    Inputs may be numpy arrays, CPU tensors or CUDA tensors; results are CUDA
    torch tensors (copies, unless copy=False gives views into the context).
    """

    def __init__(self, centres, radii, alpha: float = 0.0, opt: ac_options | None = None, offsets=None):
        self._h = None
        L = lib()
        c = _as_f64(centres)
        r = _as_f64(radii)
        n = int(r.shape[0]) if len(r.shape) else 0
        if tuple(c.shape) != (n, 3):
            raise ValueError(f"centres must be ({n}, 3), got {tuple(c.shape)}")
        self._keep = (c, r)
        h = ctypes.c_void_p()
        o = opt if opt is not None else options()
        if offsets is None:
            rc = L.ac_create(_ptr(c) if n else None, _ptr(r) if n else None, n, float(alpha), ctypes.byref(o),
                             ctypes.byref(h))
            self.n_mol = 1
        else:
            off = np.ascontiguousarray(offsets, dtype=np.int64)
            rc = L.ac_create_batch(_ptr(c) if n else None, _ptr(r) if n else None, off.ctypes.data, len(off) - 1,
                                   float(alpha), ctypes.byref(o), ctypes.byref(h))
            self.n_mol = len(off) - 1
        _check(rc, "ac_create")
        self._h = h
        self.n = n
        self.alpha = alpha

    def build(self, stream=None):
        _check(lib().ac_build(self._h, _stream_ptr(stream)), "ac_build")
        return self

    def _view(self, getter, dim, mol, width, typestr, copy):
        import torch
        p = ctypes.c_void_p()
        cnt = ctypes.c_int64()
        _check(getter(self._h, dim, mol, ctypes.byref(p), ctypes.byref(cnt)), getter.__name__)
        shape = (cnt.value, width) if width else (cnt.value,)
        if cnt.value == 0:
            dt = {"<i4": torch.int32, "<f8": torch.float64, "|u1": torch.uint8}[typestr]
            return torch.zeros(shape, dtype=dt, device="cuda")
        t = torch.as_tensor(_DeviceArray(p.value, shape, typestr), device="cuda")
        return t.clone() if copy else t

    def simplices(self, dim: int, mol: int = -1, copy: bool = True):
        return self._view(lib().ac_get_simplices, dim, mol, dim + 1, "<i4", copy)

    def filtration_values(self, dim: int, mol: int = -1, copy: bool = True):
        return self._view(lib().ac_filtration_values, dim, mol, 0, "<f8", copy)

    def attached(self, dim: int, mol: int = -1, copy: bool = True):
        return self._view(lib().ac_attached_flags, dim, mol, 0, "|u1", copy)

    def host_lists(self, dim: int, mol: int = -1, copy: bool = True):
        """(rows, filtration values, attached flags) of list dim as numpy arrays, from the host copies the
        last build made (the context needs options(host_results=True)); copy=False gives views into the
        context's page-locked memory, valid until its next build or close()."""
        t, f, a = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        cnt = ctypes.c_int64()
        _check(lib().ac_get_simplices_host(self._h, dim, mol, ctypes.byref(t), ctypes.byref(f), ctypes.byref(a),
                                           ctypes.byref(cnt)), "ac_get_simplices_host")
        n = cnt.value
        if n == 0:
            return (np.zeros((0, dim + 1), np.int32), np.zeros(0, np.float64), np.zeros(0, np.uint8))
        out = (np.ctypeslib.as_array((ctypes.c_int32 * (n * (dim + 1))).from_address(t.value)).reshape(n, dim + 1),
               np.ctypeslib.as_array((ctypes.c_double * n).from_address(f.value)),
               np.ctypeslib.as_array((ctypes.c_uint8 * n).from_address(a.value)))
        return tuple(x.copy() for x in out) if copy else out

    def candidates(self, dim: int, copy: bool = True):
        import torch
        p = ctypes.c_void_p()
        cnt = ctypes.c_int64()
        _check(lib().ac_get_candidates(self._h, dim, ctypes.byref(p), ctypes.byref(cnt)), "ac_get_candidates")
        if cnt.value == 0:
            return torch.zeros((0, dim + 1), dtype=torch.int32, device="cuda")
        t = torch.as_tensor(_DeviceArray(p.value, (cnt.value, dim + 1), "<i4"), device="cuda")
        return t.clone() if copy else t

    def autotune(self, stream=None) -> dict:
        """Time builds over cell size and block shape, keep the fastest (results unchanged)."""
        o = ac_options()
        _check(lib().ac_autotune(self._h, _stream_ptr(stream), ctypes.byref(o)), "ac_autotune")
        return {"cell_factor": o.cell_factor, "block_warps": o.block_warps}

    def subcomplex_mask(self, dim: int, alpha2: float, mol: int = -1, stream=None):
        """uint8 CUDA mask of the rows of list dim that are in K_alpha2 (alpha2 <= alpha), and their number."""
        import torch
        m = self.count(dim, mol)
        flags = torch.empty(max(m, 1), dtype=torch.uint8, device="cuda")
        cnt = ctypes.c_int64()
        _check(lib().ac_subcomplex(self._h, dim, mol, float(alpha2), flags.data_ptr(), ctypes.byref(cnt),
                                   _stream_ptr(stream)), "ac_subcomplex")
        return flags[:m], cnt.value

    def subcomplex(self, alpha2: float, mol: int = -1, stream=None):
        """The alpha complex at alpha2 <= alpha from this build: per dimension (simplices, Size values)."""
        out = []
        for d in range(4):
            mask, _ = self.subcomplex_mask(d, alpha2, mol, stream)
            keep = mask.bool()
            out.append((self.simplices(d, mol)[keep], self.filtration_values(d, mol)[keep]))
        return out

    def stats(self) -> dict:
        s = ac_stats()
        _check(lib().ac_get_stats(self._h, ctypes.byref(s)), "ac_get_stats")
        return s.to_dict()

    def eval_filtration(self, centres, radii, stream=None):
        """FP64 filtration values at other centres/radii (CUDA tensors), combinatorics fixed."""
        import torch
        c = centres.detach().to(device="cuda", dtype=torch.float64).contiguous()
        r = radii.detach().to(device="cuda", dtype=torch.float64).contiguous()
        outs = [torch.empty(self.count(d), dtype=torch.float64, device="cuda") for d in range(4)]
        ptrs = (ctypes.c_void_p * 4)(*[o.data_ptr() if o.numel() else None for o in outs])
        _check(lib().ac_eval_filtration(self._h, c.data_ptr(), r.data_ptr(), ctypes.cast(ptrs, ctypes.c_void_p),
                                        _stream_ptr(stream)), "ac_eval_filtration")
        return outs

    def eval_filtration_fp32(self, stream=None):
        """The filtration values of the last build re-evaluated in FP32 arithmetic (CUDA float32 tensors)."""
        import torch
        outs = [torch.empty(self.count(d), dtype=torch.float32, device="cuda") for d in range(4)]
        ptrs = (ctypes.c_void_p * 4)(*[o.data_ptr() if o.numel() else None for o in outs])
        _check(lib().ac_eval_filtration_fp32(self._h, ctypes.cast(ptrs, ctypes.c_void_p), _stream_ptr(stream)),
               "ac_eval_filtration_fp32")
        return outs

    def backward(self, dldf, stream=None):
        """dL/dcentres (n,3) and dL/dradii (n,) for L = sum_d dldf[d] . f[d] (CUDA float64 tensors)."""
        import torch
        ws = []
        ptrs = (ctypes.c_void_p * 4)()
        for d in range(4):
            w = None if dldf[d] is None else dldf[d].detach().to(device="cuda", dtype=torch.float64).contiguous()
            ws.append(w)
            ptrs[d] = None if (w is None or w.numel() == 0) else w.data_ptr()
        dc = torch.empty((self.n, 3), dtype=torch.float64, device="cuda")
        dr = torch.empty((self.n,), dtype=torch.float64, device="cuda")
        _check(lib().ac_backward(self._h, ctypes.cast(ptrs, ctypes.c_void_p), dc.data_ptr() if self.n else None,
                                 dr.data_ptr() if self.n else None, _stream_ptr(stream)), "ac_backward")
        return dc, dr

    def count(self, dim: int, mol: int = -1) -> int:
        p = ctypes.c_void_p()
        cnt = ctypes.c_int64()
        _check(lib().ac_get_simplices(self._h, dim, mol, ctypes.byref(p), ctypes.byref(cnt)), "ac_get_simplices")
        return cnt.value

    def close(self):
        h, self._h = self._h, None
        if h:
            lib().ac_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_f64(a, shape_tail=()):
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            raise ValueError("the chunked build takes host arrays (the molecule need not fit on the device)")
        a = a.detach().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def chunk_plan(centres, radii, alpha: float = 0.0, max_core_atoms: int = 1 << 21):
    """Slab cuts of a chunked build (host only): (thresholds int64 (k+1,), reach in quanta)."""
    c = _host_f64(centres)
    r = _host_f64(radii)
    n = int(r.shape[0])
    if c.shape != (n, 3):
        raise ValueError(f"centres must be ({n}, 3), got {c.shape}")
    k = ctypes.c_int64()
    reach = ctypes.c_int64()
    L = lib()
    rc = L.ac_chunk_plan(c.ctypes.data if n else None, r.ctypes.data if n else None, n, float(alpha),
                         int(max_core_atoms), None, 0, ctypes.byref(k), ctypes.byref(reach))
    if rc != AC_OK and rc != AC_ERR_INVALID_ARG:
        _check(rc, "ac_chunk_plan")
    thr = np.zeros(k.value + 1, dtype=np.int64)
    _check(L.ac_chunk_plan(c.ctypes.data if n else None, r.ctypes.data if n else None, n, float(alpha),
                           int(max_core_atoms), thr.ctypes.data, len(thr), ctypes.byref(k), ctypes.byref(reach)),
           "ac_chunk_plan")
    return thr[:k.value + 1] if n else thr[:0], reach.value


def _host_balls(centres, radii):
    c = _host_f64(centres)
    r = _host_f64(radii)
    n = int(r.shape[0])
    if c.shape != (n, 3):
        raise ValueError(f"centres must be ({n}, 3), got {c.shape}")
    return c, r, n


class ChunkedComplex:
    """ac_build_chunked: the alpha complex of host-resident balls, built slab by slab.

    Results are numpy arrays in host memory (copies), equal to what
    AlphaComplex gives for the whole molecule. ChunkedComplex.part gives one
    part's share (ac_build_part) and merge_parts joins shares (ac_merge_parts).
    """

    def __init__(self, centres, radii, alpha: float = 0.0, max_core_atoms: int = 1 << 21,
                 opt: ac_options | None = None, stream=None, _handle=None, _n=None):
        self._h = None
        if _handle is not None:
            self._h, self.n, self.alpha = _handle, _n, alpha
            return
        c, r, n = _host_balls(centres, radii)
        o = opt if opt is not None else options()
        h = ctypes.c_void_p()
        _check(lib().ac_build_chunked(c.ctypes.data if n else None, r.ctypes.data if n else None, n, float(alpha),
                                      ctypes.byref(o), int(max_core_atoms), _stream_ptr(stream), ctypes.byref(h)),
               "ac_build_chunked")
        self._h = h
        self.n = n
        self.alpha = alpha

    @classmethod
    def part(cls, centres, radii, alpha: float, n_parts: int, part: int, max_core_atoms: int = 1 << 21,
             opt: ac_options | None = None, stream=None):
        """ac_build_part: the rows whose first vertex lies in part `part` of n_parts z-ranges."""
        c, r, n = _host_balls(centres, radii)
        o = opt if opt is not None else options()
        h = ctypes.c_void_p()
        _check(lib().ac_build_part(c.ctypes.data if n else None, r.ctypes.data if n else None, n, float(alpha),
                                   ctypes.byref(o), int(n_parts), int(part), int(max_core_atoms), _stream_ptr(stream),
                                   ctypes.byref(h)), "ac_build_part")
        return cls(None, None, alpha, _handle=h, _n=n)

    def share(self):
        """[(rows, filtration values, attached flags)] for dimensions 0..3, numpy copies."""
        return [(self.simplices(d), self.filtration_values(d), self.attached(d)) for d in range(4)]

    def _get(self, dim):
        t, f, a = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        cnt = ctypes.c_int64()
        _check(lib().ac_chunked_simplices(self._h, dim, ctypes.byref(t), ctypes.byref(f), ctypes.byref(a),
                                          ctypes.byref(cnt)), "ac_chunked_simplices")
        return t.value, f.value, a.value, cnt.value

    @staticmethod
    def _copy(ptr, count, ctype, shape, dtype):
        if count == 0:
            return np.zeros(shape, dtype=dtype)
        buf = (ctype * int(np.prod(shape))).from_address(ptr)
        return np.frombuffer(buf, dtype=dtype).reshape(shape).copy()

    def simplices(self, dim: int):
        t, _, _, n = self._get(dim)
        return self._copy(t, n, ctypes.c_int32, (n, dim + 1), np.int32)

    def filtration_values(self, dim: int):
        _, f, _, n = self._get(dim)
        return self._copy(f, n, ctypes.c_double, (n,), np.float64)

    def attached(self, dim: int):
        _, _, a, n = self._get(dim)
        return self._copy(a, n, ctypes.c_uint8, (n,), np.uint8)

    def count(self, dim: int) -> int:
        return self._get(dim)[3]

    def stats(self) -> dict:
        st = ac_chunked_stats()
        _check(lib().ac_chunked_info(self._h, ctypes.byref(st)), "ac_chunked_info")
        return {name: getattr(st, name) for name, _ in st._fields_}

    def close(self):
        h, self._h = self._h, None
        if h:
            lib().ac_chunked_free(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def part_plan(centres, radii, alpha: float, n_parts: int):
    """ac_part_plan (host only): z thresholds (n_parts + 1, in 1/1024 A) of the parts, and the halo reach."""
    c, r, n = _host_balls(centres, radii)
    thr = np.zeros(int(n_parts) + 1, dtype=np.int64)
    reach = ctypes.c_int64()
    _check(lib().ac_part_plan(c.ctypes.data if n else None, r.ctypes.data if n else None, n, float(alpha),
                              int(n_parts), thr.ctypes.data, ctypes.byref(reach)), "ac_part_plan")
    return thr, reach.value


def merge_parts(n: int, shares, alpha: float = 0.0) -> ChunkedComplex:
    """ac_merge_parts: the whole complex from the shares of all parts (each a ChunkedComplex.share())."""
    k = len(shares)
    arrs = []
    counts = np.zeros((max(k, 1), 4), dtype=np.int64)
    tp, fp, ap = (ctypes.c_void_p * (4 * max(k, 1)))(), (ctypes.c_void_p * (4 * max(k, 1)))(), \
        (ctypes.c_void_p * (4 * max(k, 1)))()
    for p, sh in enumerate(shares):
        for d in range(4):
            t = np.ascontiguousarray(sh[d][0], dtype=np.int32).reshape(-1, d + 1)
            f = np.ascontiguousarray(sh[d][1], dtype=np.float64)
            a = np.ascontiguousarray(sh[d][2], dtype=np.uint8)
            if not (len(t) == len(f) == len(a)):
                raise ValueError(f"share {p}, dimension {d}: rows, values and flags differ in length")
            arrs += [t, f, a]
            counts[p, d] = len(t)
            tp[4 * p + d] = t.ctypes.data if len(t) else None
            fp[4 * p + d] = f.ctypes.data if len(t) else None
            ap[4 * p + d] = a.ctypes.data if len(t) else None
    h = ctypes.c_void_p()
    _check(lib().ac_merge_parts(int(n), k, counts.ctypes.data, ctypes.cast(tp, ctypes.c_void_p),
                                ctypes.cast(fp, ctypes.c_void_p), ctypes.cast(ap, ctypes.c_void_p), ctypes.byref(h)),
           "ac_merge_parts")
    return ChunkedComplex(None, None, alpha, _handle=h, _n=int(n))


def distributed_complex(centres, radii, alpha: float = 0.0, max_core_atoms: int = 1 << 21,
                        opt: ac_options | None = None, stream=None, dst: int = 0, group=None):
    """One molecule over the ranks of a torch.distributed process group (each rank on its own GPU).

    Every rank passes the whole molecule (host arrays) and builds its part
    (ac_build_part, part = rank of world size parts); the shares are gathered
    on rank dst (torch.distributed.gather_object: host memory, any backend)
    and merged there (ac_merge_parts). Returns the whole complex on dst, None
    on the other ranks. There is no other exchange: the parts are disjoint.
    """
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    mine = ChunkedComplex.part(centres, radii, alpha, world, rank, max_core_atoms, opt, stream)
    share = mine.share()
    mine.close()
    got = [None] * world if rank == dst else None
    dist.gather_object(share, got, dst=dst, group=group)
    if rank != dst:
        return None
    n = int(_host_f64(radii).shape[0])
    return merge_parts(n, got, alpha)


def fma_peak(fp64: bool = False, iters: int = 0, stream=None) -> float:
    """ac_fma_peak: the device's measured FMA throughput (FLOP/s, an FMA counts two) in FP32 or FP64."""
    if iters <= 0:
        iters = 12000 if fp64 else 800000  # about 50 ms per timed launch on one GB300
    out = ctypes.c_double()
    _check(lib().ac_fma_peak(1 if fp64 else 0, int(iters), _stream_ptr(stream), ctypes.byref(out), None),
           "ac_fma_peak")
    return out.value


def alpha_complex(centres, radii, alpha: float = 0.0, stream=None, **opt) -> AlphaComplex:
    """Create and build in one call."""
    return AlphaComplex(centres, radii, alpha, options(**opt) if opt else None).build(stream)


class AlphaFiltration:
    """torch.autograd.Function: (centres, radii) -> filtration values f[0..3] (FP64, A^2).

    The combinatorics (which simplices, and the source simplex of each value)
    are fixed by the forward build; the backward is the library's FP64 kernel.
    """

    @staticmethod
    def apply(centres, radii, alpha: float = 0.0):
        return _alpha_filtration_fn().apply(centres, radii, alpha)


_fn_cache = None


def _alpha_filtration_fn():
    global _fn_cache
    if _fn_cache is None:
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, centres, radii, alpha):
                ac = AlphaComplex(centres, radii, alpha).build()
                ctx.ac = ac
                ctx.dtypes = (centres.dtype, radii.dtype, centres.device)
                return tuple(ac.filtration_values(d) for d in range(4))

            @staticmethod
            def backward(ctx, *grads):
                dc, dr = ctx.ac.backward(list(grads))
                cdt, rdt, dev = ctx.dtypes
                return dc.to(device=dev, dtype=cdt), dr.to(device=dev, dtype=rdt), None

        _fn_cache = _F
    return _fn_cache
