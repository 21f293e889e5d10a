"""ORACLE - TEST INFRASTRUCTURE ONLY.

ctypes binding of oracle.c, the plain single-threaded CPU statement of
FastCod's pass-through connectivity (arXiv 2302.09247, Section 2, Algorithms
1-2).  Only the tests, the package smoke check and the benchmark's CPU-baseline
leg import this module; the CUDA library never does.  It shares no code with
the CUDA path.

Pinned by tests/test_oracle_*.py against brute force (exact slab tests), closed
forms, invariants and a library matrix product; no function here is "parity
unpinned" except agreement with real tractography data, which is not in scope.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

TARGET_ENDPOINT = 1
VERTEX_SAMPLED = 2


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(src),
                                                                          os.path.getmtime(hdr)):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, src,
                               "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Stats(ctypes.Structure):
    _fields_ = [("voxel_steps", ctypes.c_int64), ("visits", ctypes.c_int64),
                ("n_contributing", ctypes.c_int64), ("pairs", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        L.oracle_segment_voxels.restype = i64
        L.oracle_segment_voxels.argtypes = [vp, vp, vp, i64]
        L.oracle_bruteforce_segment.restype = i64
        L.oracle_bruteforce_segment.argtypes = [vp, vp, vp, vp, vp, i64]
        L.oracle_connectivity.restype = ctypes.c_int
        L.oracle_connectivity.argtypes = [vp, vp, vp, i32, i32, vp, vp, i64, u32, vp, vp,
                                          ctypes.POINTER(Stats)]
        L.oracle_bruteforce_connectivity.restype = ctypes.c_int
        L.oracle_bruteforce_connectivity.argtypes = [vp, vp, vp, i32, i32, vp, vp, i64, u32, vp, vp]
        L.oracle_streamline_sets.restype = ctypes.c_int
        L.oracle_streamline_sets.argtypes = [vp, vp, vp, i32, i32, vp, i64, u32, vp, vp, vp, vp]
        L.oracle_parcellate.restype = ctypes.c_int
        L.oracle_parcellate.argtypes = [vp, i32, i32, vp, vp]
        L.oracle_world_to_fixed.restype = ctypes.c_int
        L.oracle_world_to_fixed.argtypes = [vp, i64, vp, vp]
        L.oracle_upsample.restype = i64
        L.oracle_upsample.argtypes = [vp, vp, i64, i32, vp, vp]
        L.oracle_upsample_factor.restype = i32
        L.oracle_upsample_factor.argtypes = [vp, vp, i64, i32]
        L.oracle_rescale.restype = ctypes.c_int
        L.oracle_rescale.argtypes = [vp, i64, vp, vp, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _i32x3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(3))


def segment_voxels(p0, p1) -> np.ndarray:
    """Voxels visited by the walk of segment p0 -> p1 (1/1024-voxel units), in order."""
    a, b = _i32x3(p0), _i32x3(p1)
    cap = 64
    while True:
        out = np.empty((cap, 3), dtype=np.int32)
        n = lib().oracle_segment_voxels(_p(a), _p(b), _p(out), cap)
        if n <= cap:
            return out[:n].copy()
        cap = int(n)


def bruteforce_segment(p0, p1, lo, hi) -> np.ndarray:
    """Voxels in the inclusive box [lo, hi] whose half-open box meets the closed segment."""
    a, b, l, h = _i32x3(p0), _i32x3(p1), _i32x3(lo), _i32x3(hi)
    cap = int(np.prod(h.astype(np.int64) - l + 1))
    out = np.empty((max(cap, 1), 3), dtype=np.int32)
    n = lib().oracle_bruteforce_segment(_p(a), _p(b), _p(l), _p(h), _p(out), cap)
    return out[:n].copy()


def _vol_args(roi, lab, dims):
    roi = np.ascontiguousarray(roi, dtype=np.int32)
    lab = np.ascontiguousarray(lab, dtype=np.uint16)
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(3))
    assert roi.size == lab.size == int(np.prod(d.astype(np.int64)))
    return roi, lab, d


def connectivity(roi, lab, dims, N, M, xyz, offsets, flags: int = 0, with_end: bool = True):
    """(C, C_end, stats) with int64 C, C_end of shape (N, M)."""
    roi, lab, d = _vol_args(roi, lab, dims)
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    C = np.zeros((N, M), dtype=np.int64)
    Ce = np.zeros((N, M), dtype=np.int64) if with_end else None
    st = Stats()
    rc = lib().oracle_connectivity(_p(roi), _p(lab), _p(d), N, M, _p(xyz), _p(off), len(off) - 1,
                                   flags, _p(C), _p(Ce), ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle: invalid input")
    return C, Ce, st.as_dict()


def connectivity_chunked(roi, lab, dims, N, M, xyz, offsets, flags: int = 0, threads: int | None = None,
                         chunks: int | None = None):
    """The same result as connectivity(), computed on contiguous streamline
    chunks in threads and summed (integer addition is exact and associative).
    ctypes releases the GIL during each oracle call."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ns = len(off) - 1
    threads = threads or max(1, min(32, os.cpu_count() or 1))
    chunks = chunks or threads * 4
    bounds = np.linspace(0, ns, chunks + 1).astype(np.int64)

    def run(k):
        b, e = int(bounds[k]), int(bounds[k + 1])
        o = off[b:e + 1] - off[b]
        return connectivity(roi, lab, dims, N, M, xyz[off[b]:off[e]], o, flags)

    C = np.zeros((N, M), dtype=np.int64)
    Ce = np.zeros((N, M), dtype=np.int64)
    st = {"voxel_steps": 0, "visits": 0, "n_contributing": 0, "pairs": 0}
    with ThreadPoolExecutor(threads) as ex:
        for c, ce, s in ex.map(run, range(chunks)):
            C += c
            Ce += ce
            for k in st:
                st[k] += s[k]
    return C, Ce, st


def bruteforce_connectivity(roi, lab, dims, N, M, xyz, offsets, flags: int = 0):
    roi, lab, d = _vol_args(roi, lab, dims)
    xyz = np.ascontiguousarray(xyz, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    C = np.zeros((N, M), dtype=np.int64)
    Ce = np.zeros((N, M), dtype=np.int64)
    rc = lib().oracle_bruteforce_connectivity(_p(roi), _p(lab), _p(d), N, M, _p(xyz), _p(off),
                                              len(off) - 1, flags, _p(C), _p(Ce))
    if rc != 0:
        raise ValueError("oracle: invalid input")
    return C, Ce


def streamline_sets(roi, lab, dims, N, M, verts, flags: int = 0):
    """(V_s, T_s) of one streamline, each sorted ascending."""
    roi, lab, d = _vol_args(roi, lab, dims)
    v = np.ascontiguousarray(verts, dtype=np.int32).reshape(-1, 3)
    V = np.empty(max(N, 1), dtype=np.int32)
    Tl = np.empty(M + 1, dtype=np.int32)
    nV, nT = ctypes.c_int32(), ctypes.c_int32()
    lib().oracle_streamline_sets(_p(roi), _p(lab), _p(d), N, M, _p(v), len(v), flags, _p(V),
                                 ctypes.byref(nV), _p(Tl), ctypes.byref(nT))
    return V[:nV.value].copy(), Tl[:nT.value].copy()


def parcellate(C):
    """(label int32 [N], fractions float32 [N, M]) of a connectivity matrix
    (Section 3, pie-glyphs and the single-colour display)."""
    C = np.ascontiguousarray(C, dtype=np.int64)
    N, M = C.shape
    label = np.empty(N, dtype=np.int32)
    frac = np.empty((N, M), dtype=np.float32)
    rc = lib().oracle_parcellate(_p(C), N, M, _p(label), _p(frac))
    if rc != 0:
        raise ValueError("oracle: negative count" if rc == -1 else "oracle: row sum reaches 2^62")
    return label, frac


def world_to_fixed(xyz_mm, affine):
    """int32 fixed-point vertices from binary32 world-mm vertices and a 3x4
    world -> voxel affine (binary32)."""
    x = np.ascontiguousarray(xyz_mm, dtype=np.float32).reshape(-1, 3)
    A = np.ascontiguousarray(affine, dtype=np.float32).reshape(12)
    out = np.empty(x.shape, dtype=np.int32)
    if lib().oracle_world_to_fixed(_p(x), len(x), _p(A), _p(out)) != 0:
        raise ValueError("oracle: coordinate not finite or out of range")
    return out


def upsample(xyz, offsets, factor: int):
    """(xyz, offsets) with `factor` segments per original segment."""
    xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ns = len(off) - 1
    nonempty = int(np.count_nonzero(np.diff(off)))
    nv_out = (len(xyz) - nonempty) * factor + nonempty
    out = np.empty((max(nv_out, 0), 3), dtype=np.int32)
    oo = np.empty(ns + 1, dtype=np.int64)
    n = lib().oracle_upsample(_p(xyz), _p(off), ns, int(factor), _p(out), _p(oo))
    if n < 0:
        raise ValueError("oracle: invalid input")
    assert n == nv_out
    return out, oo


def upsample_factor(xyz, offsets, spacing: int) -> int:
    xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    k = lib().oracle_upsample_factor(_p(xyz), _p(off), len(off) - 1, int(spacing))
    if k < 0:
        raise ValueError("oracle: invalid input")
    return int(k)


def rescale(xyz, num, den, add):
    xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    num = np.ascontiguousarray(num, dtype=np.int32)
    den = np.ascontiguousarray(den, dtype=np.int32)
    add = np.ascontiguousarray(add, dtype=np.int64)
    out = np.empty_like(xyz)
    if lib().oracle_rescale(_p(xyz), len(xyz), _p(num), _p(den), _p(add), _p(out)) != 0:
        raise ValueError("oracle: invalid input or result out of range")
    return out
