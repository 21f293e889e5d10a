"""Thin ctypes binding of libfastcod (include/fastcod.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names; array arguments may be numpy arrays
(host memory), torch tensors (host, pinned or CUDA) or raw integer addresses.
There is no CPU fallback: importing this module fails loudly when the library
has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FASTCOD_LIBRARY overrides the in-tree build (e.g. a custom build of the same sources)
LIB_PATH = os.environ.get("FASTCOD_LIBRARY") or os.path.join(_HERE, "_lib", "libfastcod.so")

FASTCOD_OK = 0
FASTCOD_EINVAL = -1
FASTCOD_ENOMEM = -2
FASTCOD_ECUDA = -3
FASTCOD_ESTATE = -4
FASTCOD_EOVERFLOW = -5
FASTCOD_ETIMEOUT = -6
FASTCOD_ECANCELED = -7

FASTCOD_SYNC = 1

FASTCOD_OPT_PREFILTER = 1
FASTCOD_OPT_TARGET_MODE = 2
FASTCOD_OPT_SAMPLING = 3
FASTCOD_OPT_STAGING = 4
FASTCOD_OPT_PROFILE = 5
FASTCOD_OPT_PREFILTER_CTAS = 6
FASTCOD_OPT_NEAR_LOG2 = 7
FASTCOD_OPT_AUTOTUNE = 8
FASTCOD_OPT_HOST_IN_PLACE = 9
FASTCOD_OPT_WALKED_STEPS = 10
FASTCOD_OPT_SEGMENT_SKIP = 11
FASTCOD_OPT_TEST_WITHHOLD_PIECE = 12
FASTCOD_OPT_BATCH_TASK_LOG2 = 13

EXPORTED = [
    "fastcod_create", "fastcod_destroy", "fastcod_set_stream", "fastcod_set_volumes",
    "fastcod_add_streamlines", "fastcod_connectivity", "fastcod_endpoint_connectivity",
    "fastcod_reset", "fastcod_get_shape", "fastcod_get_stats", "fastcod_restore", "fastcod_get_profile",
    "fastcod_sync",
    "fastcod_set_option", "fastcod_last_error", "fastcod_batch_run", "fastcod_batch_get_stats",
    "fastcod_batch_get_info", "fastcod_server_create", "fastcod_server_submit", "fastcod_server_push_chunk",
    "fastcod_server_poll", "fastcod_server_wait", "fastcod_server_cancel", "fastcod_server_request_info",
    "fastcod_server_destroy", "fastcod_server_kernel_launches", "fastcod_connectivity_noalloc", "fastcod_parcellate", "fastcod_parcellate_matrix",
    "fastcod_world_to_fixed",
    "fastcod_add_streamlines_mm", "fastcod_upsample", "fastcod_upsample_factor", "fastcod_rescale",
]


class FastCodError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fastcod error {code}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("streamlines", ctypes.c_int64), ("vertices", ctypes.c_int64),
                ("voxel_steps", ctypes.c_int64), ("survivors", ctypes.c_int64),
                ("overflow", ctypes.c_int64), ("pairs", ctypes.c_int64), ("walked_steps", ctypes.c_int64)]


class Profile(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("ms_h2d", ctypes.c_double),
                ("ms_prefilter", ctypes.c_double), ("ms_walk", ctypes.c_double),
                ("ms_overflow", ctypes.c_double), ("aux_calls", ctypes.c_int64), ("ms_aux", ctypes.c_double)]


class Subject(ctypes.Structure):
    _fields_ = [("roi_index_map", ctypes.c_void_p), ("target_labels", ctypes.c_void_p),
                ("dims", ctypes.c_int32 * 3), ("n_roi", ctypes.c_int32), ("n_targets", ctypes.c_int32),
                ("xyz", ctypes.c_void_p), ("n_vertices", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("n_streamlines", ctypes.c_int64), ("C_out", ctypes.c_void_p), ("Cend_out", ctypes.c_void_p)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_subjects", ctypes.c_int32), ("tasks", ctypes.c_int32), ("prefilter_ctas", ctypes.c_int32),
                ("near_log2", ctypes.c_int32), ("graph_reused", ctypes.c_int32), ("tuned", ctypes.c_int32),
                ("ms_graph", ctypes.c_double), ("task_vertices", ctypes.c_int64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("done", ctypes.c_int32), ("streamlines", ctypes.c_int64),
                ("chunks", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2302_09247_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "fastcod_create": ([ctypes.POINTER(vp), ctypes.c_int, u32], ctypes.c_int),
        "fastcod_destroy": ([vp], ctypes.c_int),
        "fastcod_set_stream": ([vp, vp], ctypes.c_int),
        "fastcod_set_volumes": ([vp, vp, vp, i32, i32, i32, i32, i32], ctypes.c_int),
        "fastcod_add_streamlines": ([vp, vp, i64, vp, i64], ctypes.c_int),
        "fastcod_connectivity": ([vp, vp], ctypes.c_int),
        "fastcod_endpoint_connectivity": ([vp, vp], ctypes.c_int),
        "fastcod_reset": ([vp], ctypes.c_int),
        "fastcod_get_shape": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
        "fastcod_get_stats": ([vp, ctypes.POINTER(Stats)], ctypes.c_int),
        "fastcod_restore": ([vp, vp, vp, ctypes.POINTER(Stats)], ctypes.c_int),
        "fastcod_get_profile": ([vp, ctypes.POINTER(Profile)], ctypes.c_int),
        "fastcod_sync": ([vp], ctypes.c_int),
        "fastcod_set_option": ([vp, i32, i64], ctypes.c_int),
        "fastcod_last_error": ([vp], ctypes.c_char_p),
        "fastcod_batch_run": ([vp, ctypes.POINTER(Subject), i32], ctypes.c_int),
        "fastcod_batch_get_stats": ([vp, i32, ctypes.POINTER(Stats)], ctypes.c_int),
        "fastcod_batch_get_info": ([vp, ctypes.POINTER(BatchInfo)], ctypes.c_int),
        "fastcod_server_create": ([vp, i32, i64, ctypes.POINTER(vp)], ctypes.c_int),
        "fastcod_server_submit": ([vp, ctypes.POINTER(Subject), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "fastcod_server_push_chunk": ([vp, ctypes.c_uint64, vp, i64, vp, i64, i32], ctypes.c_int),
        "fastcod_server_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(i32)], ctypes.c_int),
        "fastcod_server_wait": ([vp, ctypes.c_uint64, ctypes.c_double], ctypes.c_int),
        "fastcod_server_cancel": ([vp, ctypes.c_uint64], ctypes.c_int),
        "fastcod_server_request_info": ([vp, ctypes.c_uint64, ctypes.POINTER(RequestInfo)], ctypes.c_int),
        "fastcod_server_kernel_launches": ([vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "fastcod_server_destroy": ([vp], ctypes.c_int),
        "fastcod_connectivity_noalloc": ([ctypes.c_int, vp, vp, vp, i32, i32, i32, i32, i32, vp, i64, vp, i64, vp,
                                          vp], ctypes.c_int),
        "fastcod_parcellate": ([vp, i32, vp, vp], ctypes.c_int),
        "fastcod_parcellate_matrix": ([vp, vp, i32, i32, vp, vp], ctypes.c_int),
        "fastcod_world_to_fixed": ([vp, vp, i64, vp, vp], ctypes.c_int),
        "fastcod_add_streamlines_mm": ([vp, vp, i64, vp, i64, vp], ctypes.c_int),
        "fastcod_upsample": ([vp, vp, i64, vp, i64, i32, vp, i64, vp], ctypes.c_int),
        "fastcod_upsample_factor": ([vp, vp, i64, vp, i64, i32, ctypes.POINTER(i32)], ctypes.c_int),
        "fastcod_rescale": ([vp, vp, i64, vp, vp, vp, vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def _ptr(x):
    """Address of a contiguous numpy array / torch tensor, or an int address."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(ctx, rc):
    if rc != FASTCOD_OK:
        raise FastCodError(rc, lib.fastcod_last_error(ctx).decode())
    return rc


def fastcod_create(device: int = 0, flags: int = 0):
    out = ctypes.c_void_p()
    rc = lib.fastcod_create(ctypes.byref(out), device, flags)
    if rc != FASTCOD_OK:
        raise FastCodError(rc, lib.fastcod_last_error(None).decode())
    return out


def fastcod_destroy(ctx):
    return lib.fastcod_destroy(ctx)


def fastcod_set_stream(ctx, stream):
    s = getattr(stream, "cuda_stream", stream)
    return _check(ctx, lib.fastcod_set_stream(ctx, s))


def fastcod_set_volumes(ctx, roi, lab, dims, n_roi: int = 0, n_targets: int = 0):
    dx, dy, dz = (int(d) for d in dims)
    return _check(ctx, lib.fastcod_set_volumes(ctx, _ptr(roi), _ptr(lab), dx, dy, dz, n_roi, n_targets))


def fastcod_add_streamlines(ctx, xyz, offsets, n_vertices: int | None = None, n_streamlines: int | None = None):
    nv = int(xyz.shape[0]) if n_vertices is None else int(n_vertices)
    ns = int(offsets.shape[0]) - 1 if n_streamlines is None else int(n_streamlines)
    return _check(ctx, lib.fastcod_add_streamlines(ctx, _ptr(xyz), nv, _ptr(offsets), ns))


def fastcod_connectivity(ctx, out):
    return _check(ctx, lib.fastcod_connectivity(ctx, _ptr(out)))


def fastcod_endpoint_connectivity(ctx, out):
    return _check(ctx, lib.fastcod_endpoint_connectivity(ctx, _ptr(out)))


def fastcod_reset(ctx):
    return _check(ctx, lib.fastcod_reset(ctx))


def fastcod_get_shape(ctx):
    n, m = ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, lib.fastcod_get_shape(ctx, ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def fastcod_get_stats(ctx) -> dict:
    s = Stats()
    _check(ctx, lib.fastcod_get_stats(ctx, ctypes.byref(s)))
    return {k: int(getattr(s, k)) for k, _ in Stats._fields_}


def fastcod_restore(ctx, C, Cend, stats: dict):
    """Install a checkpoint: C and C_end (int32 [N][M], host or device) and the
    statistics dict fastcod_get_stats returned when they were read."""
    s = Stats(**{k: int(stats[k]) for k, _ in Stats._fields_})
    return _check(ctx, lib.fastcod_restore(ctx, _ptr(C), _ptr(Cend), ctypes.byref(s)))


def fastcod_get_profile(ctx) -> dict:
    p = Profile()
    _check(ctx, lib.fastcod_get_profile(ctx, ctypes.byref(p)))
    return {k: (float(getattr(p, k)) if k.startswith("ms_") else int(getattr(p, k))) for k, _ in Profile._fields_}


def fastcod_sync(ctx):
    return _check(ctx, lib.fastcod_sync(ctx))


def fastcod_set_option(ctx, key: int, value: int):
    return _check(ctx, lib.fastcod_set_option(ctx, key, value))


def fastcod_last_error(ctx) -> str:
    return lib.fastcod_last_error(ctx).decode()


def make_subject(roi, lab, dims, n_roi, n_targets, xyz, offsets, C_out, Cend_out) -> Subject:
    """A fastcod_subject from arrays / tensors (the caller keeps them alive)."""
    s = Subject()
    s.roi_index_map = _ptr(roi)
    s.target_labels = _ptr(lab)
    for a in range(3):
        s.dims[a] = int(dims[a])
    s.n_roi = int(n_roi)
    s.n_targets = int(n_targets)
    s.xyz = _ptr(xyz)
    s.n_vertices = int(xyz.shape[0])
    s.offsets = _ptr(offsets)
    s.n_streamlines = int(offsets.shape[0]) - 1
    s.C_out = _ptr(C_out)
    s.Cend_out = _ptr(Cend_out)
    return s


def fastcod_batch_run(ctx, subjects):
    arr = (Subject * len(subjects))(*subjects)
    return _check(ctx, lib.fastcod_batch_run(ctx, arr, len(subjects)))


def fastcod_batch_get_stats(ctx, subject: int) -> dict:
    st = Stats()
    _check(ctx, lib.fastcod_batch_get_stats(ctx, subject, ctypes.byref(st)))
    return {k: int(getattr(st, k)) for k, _ in Stats._fields_}


def fastcod_batch_get_info(ctx) -> dict:
    info = BatchInfo()
    _check(ctx, lib.fastcod_batch_get_info(ctx, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in BatchInfo._fields_}


def fastcod_server_create(ctx, max_slots: int = 8, hbm_budget_bytes: int = 0):
    out = ctypes.c_void_p()
    _check(ctx, lib.fastcod_server_create(ctx, max_slots, hbm_budget_bytes, ctypes.byref(out)))
    return out


def _scheck(rc):
    if rc != FASTCOD_OK:
        raise FastCodError(rc, "server call failed")
    return rc


def fastcod_server_submit(srv, head: Subject) -> int:
    rid = ctypes.c_uint64()
    _scheck(lib.fastcod_server_submit(srv, ctypes.byref(head), ctypes.byref(rid)))
    return rid.value


def fastcod_server_push_chunk(srv, rid: int, xyz, offsets, last: bool = False):
    if xyz is None:
        return _scheck(lib.fastcod_server_push_chunk(srv, rid, None, 0, None, 0, 1 if last else 0))
    return _scheck(lib.fastcod_server_push_chunk(srv, rid, _ptr(xyz), int(xyz.shape[0]), _ptr(offsets),
                                                 int(offsets.shape[0]) - 1, 1 if last else 0))


def fastcod_server_poll(srv, rid: int):
    """(done, status)"""
    done = ctypes.c_int32()
    rc = lib.fastcod_server_poll(srv, rid, ctypes.byref(done))
    return bool(done.value), rc


def fastcod_server_wait(srv, rid: int, timeout_s: float = 60.0) -> int:
    """The request's status (FASTCOD_ETIMEOUT if it did not finish in time)."""
    return lib.fastcod_server_wait(srv, rid, timeout_s)


def fastcod_server_cancel(srv, rid: int):
    return _scheck(lib.fastcod_server_cancel(srv, rid))


def fastcod_server_request_info(srv, rid: int) -> dict:
    info = RequestInfo()
    _scheck(lib.fastcod_server_request_info(srv, rid, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in RequestInfo._fields_}


def fastcod_server_kernel_launches(srv) -> int:
    n = ctypes.c_int64()
    _scheck(lib.fastcod_server_kernel_launches(srv, ctypes.byref(n)))
    return int(n.value)


def fastcod_server_destroy(srv):
    return lib.fastcod_server_destroy(srv)


def fastcod_connectivity_noalloc(device, stream, roi, lab, dims, n_roi, n_targets, xyz, offsets, C_out, Cend_out):
    """The allocation-free entry point: every array is device memory."""
    s = getattr(stream, "cuda_stream", stream)
    dx, dy, dz = (int(d) for d in dims)
    rc = lib.fastcod_connectivity_noalloc(device, s, _ptr(roi), _ptr(lab), dx, dy, dz, int(n_roi), int(n_targets),
                                          _ptr(xyz), int(xyz.shape[0]), _ptr(offsets), int(offsets.shape[0]) - 1,
                                          _ptr(C_out), _ptr(Cend_out))
    if rc != FASTCOD_OK:
        raise FastCodError(rc, lib.fastcod_last_error(None).decode())
    return rc


def fastcod_parcellate(ctx, which: int, label_out, fractions_out=None):
    return _check(ctx, lib.fastcod_parcellate(ctx, int(which), _ptr(label_out), _ptr(fractions_out)))


def fastcod_parcellate_matrix(ctx, C, label_out, fractions_out=None):
    """Parcellation outputs of a caller's int32 [N, M] matrix (host or device)."""
    if str(C.dtype) not in ("int32", "torch.int32") or len(C.shape) != 2:
        raise TypeError("C must be a 2-D int32 array or tensor")
    N, M = (int(d) for d in C.shape)
    return _check(ctx, lib.fastcod_parcellate_matrix(ctx, _ptr(C), N, M, _ptr(label_out), _ptr(fractions_out)))


def _affine(affine):
    a = np.ascontiguousarray(np.asarray(affine, dtype=np.float32).reshape(-1)[:12])
    if a.size != 12:
        raise ValueError("affine needs 12 values (3 x 4, row-major)")
    return a


def fastcod_world_to_fixed(ctx, xyz_mm, affine, xyz_out):
    a = _affine(affine)
    return _check(ctx, lib.fastcod_world_to_fixed(ctx, _ptr(xyz_mm), int(xyz_mm.shape[0]), a.ctypes.data,
                                                  _ptr(xyz_out)))


def fastcod_add_streamlines_mm(ctx, xyz_mm, offsets, affine):
    a = _affine(affine)
    return _check(ctx, lib.fastcod_add_streamlines_mm(ctx, _ptr(xyz_mm), int(xyz_mm.shape[0]), _ptr(offsets),
                                                      int(offsets.shape[0]) - 1, a.ctypes.data))


def upsampled_count(offsets_host: np.ndarray, factor: int) -> int:
    """Vertices of the upsampled tractogram (host offsets)."""
    T = np.diff(np.asarray(offsets_host, dtype=np.int64))
    nonempty = int(np.count_nonzero(T))
    return (int(T.sum()) - nonempty) * int(factor) + nonempty


def fastcod_upsample(ctx, xyz, offsets, factor: int, xyz_out, offsets_out):
    return _check(ctx, lib.fastcod_upsample(ctx, _ptr(xyz), int(xyz.shape[0]), _ptr(offsets),
                                            int(offsets.shape[0]) - 1, int(factor), _ptr(xyz_out),
                                            int(xyz_out.shape[0]), _ptr(offsets_out)))


def fastcod_upsample_factor(ctx, xyz, offsets, spacing: int) -> int:
    k = ctypes.c_int32()
    _check(ctx, lib.fastcod_upsample_factor(ctx, _ptr(xyz), int(xyz.shape[0]), _ptr(offsets),
                                           int(offsets.shape[0]) - 1, int(spacing), ctypes.byref(k)))
    return int(k.value)


def fastcod_rescale(ctx, xyz, num, den, add, xyz_out):
    n = np.ascontiguousarray(num, dtype=np.int32)
    d = np.ascontiguousarray(den, dtype=np.int32)
    a = np.ascontiguousarray(add, dtype=np.int64)
    return _check(ctx, lib.fastcod_rescale(ctx, _ptr(xyz), int(xyz.shape[0]), n.ctypes.data, d.ctypes.data,
                                           a.ctypes.data, _ptr(xyz_out)))


class Context:
    """Convenience owner of a fastcod context."""

    def __init__(self, device: int = 0, flags: int = 0):
        self.ctx = fastcod_create(device, flags)

    def close(self):
        if self.ctx is not None:
            fastcod_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_volumes(self, roi, lab, dims, n_roi: int = 0, n_targets: int = 0):
        fastcod_set_volumes(self.ctx, roi, lab, dims, n_roi, n_targets)
        return self.shape()

    def add_streamlines(self, xyz, offsets):
        fastcod_add_streamlines(self.ctx, xyz, offsets)

    def shape(self):
        return fastcod_get_shape(self.ctx)

    def connectivity(self, out=None):
        if out is None:
            n, m = self.shape()
            out = np.empty((n, m), dtype=np.int32)
        fastcod_connectivity(self.ctx, out)
        return out

    def endpoint_connectivity(self, out=None):
        if out is None:
            n, m = self.shape()
            out = np.empty((n, m), dtype=np.int32)
        fastcod_endpoint_connectivity(self.ctx, out)
        return out

    def stats(self) -> dict:
        return fastcod_get_stats(self.ctx)

    def checkpoint(self):
        """(C, C_end, statistics) as host arrays and a dict."""
        return self.connectivity(), self.endpoint_connectivity(), self.stats()

    def restore(self, C, Cend, stats: dict):
        fastcod_restore(self.ctx, C, Cend, stats)

    def profile(self) -> dict:
        return fastcod_get_profile(self.ctx)

    def set_option(self, key: int, value: int):
        fastcod_set_option(self.ctx, key, value)

    def reset(self):
        fastcod_reset(self.ctx)

    def sync(self):
        fastcod_sync(self.ctx)
