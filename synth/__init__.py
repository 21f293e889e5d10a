"""Seeded synthetic inputs: volumes and tractograms (ctypes over synth.c).

Shared by the CUDA path's tests, the oracle's tests and the benchmark; it holds
none of the connectivity method's arithmetic (no voxel walk, no counting).

The five workload presets stand in for the paper's HCP data (Section 3): an
ellipsoidal brain, thalamus-like ROI ellipsoids, an M-way angular Voronoi
cortical shell and persistent random-walk streamlines.

    cfg0  tiny       32^3 @ 1 mm,   one ROI ellipsoid (~200 vox), M=8,   20,000 streamlines
    cfg1  HCP-shaped 145x174x145 @ 1.25 mm, two thalami (N~7,000), M=70, 2,000,000 streamlines
    cfg2  high-res   260x311x260 @ 0.7 mm,  two thalami (N~40,000), M=360, 5,000,000 streamlines
    cfg3  batched    64 subjects, grids 96^3..145x174x145, M in {8,70,360}, N 1,000..12,000
    cfg4  served     cfg1-shaped subjects, 200,000..2,000,000 streamlines per request
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsynth.so")

# Fraction of seeds placed inside ROI voxels.  Chosen once so that about 10%
# of the HCP-shaped (cfg1) streamlines pass through the thalamus.
F_ROI = 0.065


def build(force: bool = False) -> str:
    """Compile synth.c into _build/libsynth.so (gcc, portable flags)."""
    src = os.path.join(_HERE, "synth.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "synth.h"))
    ):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
             "-o", tmp, src, "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


class _VolParams(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int32 * 3),
        ("brain_c", ctypes.c_double * 3),
        ("brain_ax", ctypes.c_double * 3),
        ("shell_rho_in", ctypes.c_double),
        ("n_labels", ctypes.c_int32),
        ("label_seed", ctypes.c_uint64),
        ("n_roi", ctypes.c_int32),
        ("roi_c", (ctypes.c_double * 3) * 4),
        ("roi_ax", (ctypes.c_double * 3) * 4),
    ]


class _SlParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("subject", ctypes.c_uint32),
        ("step_vox", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("len_mode", ctypes.c_int32),
        ("len_a", ctypes.c_double),
        ("len_b", ctypes.c_double),
        ("len_sigma", ctypes.c_double),
        ("len_lo", ctypes.c_double),
        ("len_hi", ctypes.c_double),
        ("res_mm", ctypes.c_double),
        ("f_roi", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        _lib.synth_volumes.restype = ctypes.c_int64
        _lib.synth_volumes.argtypes = [P(_VolParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        _lib.synth_count.restype = ctypes.c_int
        _lib.synth_count.argtypes = [P(_VolParams), P(_SlParams), ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32]
        _lib.synth_fill.restype = ctypes.c_int
        _lib.synth_fill.argtypes = [P(_VolParams), P(_SlParams), ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int32]
        _lib.synth_splitmix64.restype = None
        _lib.synth_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64]
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def n_threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def splitmix64(state: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    lib().synth_splitmix64(ctypes.c_uint64(state), _ptr(out), n)
    return out


@dataclass
class VolumeSpec:
    dims: tuple                       # (Dx, Dy, Dz)
    brain_c: tuple                    # voxel units
    brain_ax: tuple                   # voxel units
    shell_rho_in: float
    n_labels: int
    label_seed: int
    roi_c: list = field(default_factory=list)   # list of (x, y, z) voxel units
    roi_ax: list = field(default_factory=list)  # list of (a, b, c) voxel units

    def _c(self) -> _VolParams:
        p = _VolParams()
        for a in range(3):
            p.dims[a] = int(self.dims[a])
            p.brain_c[a] = float(self.brain_c[a])
            p.brain_ax[a] = float(self.brain_ax[a])
        p.shell_rho_in = float(self.shell_rho_in)
        p.n_labels = int(self.n_labels)
        p.label_seed = int(self.label_seed)
        p.n_roi = len(self.roi_c)
        for e, (c, ax) in enumerate(zip(self.roi_c, self.roi_ax)):
            for a in range(3):
                p.roi_c[e][a] = float(c[a])
                p.roi_ax[e][a] = float(ax[a])
        return p


@dataclass
class StreamlineSpec:
    n_streamlines: int
    seed: int
    subject: int = 0
    step_vox: float = 0.5
    kappa: float = 20.0
    len_mode: int = 0          # 0: uniform vertices [len_a, len_b]; 1: lognormal mm
    len_a: float = 20
    len_b: float = 120
    len_sigma: float = 0.5
    len_lo: float = 20.0
    len_hi: float = 250.0
    res_mm: float = 1.0
    f_roi: float = F_ROI

    def _c(self) -> _SlParams:
        p = _SlParams()
        p.seed = int(self.seed)
        p.subject = int(self.subject)
        p.step_vox = float(self.step_vox)
        p.kappa = float(self.kappa)
        p.len_mode = int(self.len_mode)
        p.len_a = float(self.len_a)
        p.len_b = float(self.len_b)
        p.len_sigma = float(self.len_sigma)
        p.len_lo = float(self.len_lo)
        p.len_hi = float(self.len_hi)
        p.res_mm = float(self.res_mm)
        p.f_roi = float(self.f_roi)
        return p


@dataclass
class Volumes:
    roi: np.ndarray      # int32 [Dz, Dy, Dx], -1 outside, else row index
    lab: np.ndarray      # uint16 [Dz, Dy, Dx], 0 = no target
    dims: tuple          # (Dx, Dy, Dz)
    n_roi: int           # N
    n_targets: int       # M
    roi_lin: np.ndarray  # int64 linear indices of ROI voxels (seed pool)


@dataclass
class Tractogram:
    xyz: np.ndarray      # int32 [nv, 3], 1/1024 voxel
    offsets: np.ndarray  # int64 [ns + 1]

    @property
    def n_streamlines(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_vertices(self) -> int:
        return int(self.offsets[-1])


def make_volumes(vs: VolumeSpec, threads: int | None = None) -> Volumes:
    Dx, Dy, Dz = (int(d) for d in vs.dims)
    roi = np.empty((Dz, Dy, Dx), dtype=np.int32)
    lab = np.empty((Dz, Dy, Dx), dtype=np.uint16)
    p = vs._c()
    n = lib().synth_volumes(ctypes.byref(p), _ptr(roi), _ptr(lab), threads or n_threads())
    if n < 0:
        raise ValueError("invalid volume parameters")
    roi_lin = np.flatnonzero(roi.reshape(-1) >= 0).astype(np.int64)
    return Volumes(roi, lab, (Dx, Dy, Dz), int(n), int(vs.n_labels), roi_lin)


def count_vertices(vs: VolumeSpec, ss: StreamlineSpec, vols: Volumes, s_begin: int = 0,
                   s_end: int | None = None, threads: int | None = None) -> np.ndarray:
    s_end = ss.n_streamlines if s_end is None else s_end
    counts = np.empty(s_end - s_begin, dtype=np.int32)
    vp, sp = vs._c(), ss._c()
    rl = np.ascontiguousarray(vols.roi_lin)
    lib().synth_count(ctypes.byref(vp), ctypes.byref(sp), _ptr(rl), len(rl), s_begin, s_end,
                      _ptr(counts), threads or n_threads())
    return counts


def fill_vertices(vs: VolumeSpec, ss: StreamlineSpec, vols: Volumes, offsets: np.ndarray,
                  xyz_ptr: int, s_begin: int = 0, s_end: int | None = None,
                  threads: int | None = None) -> None:
    """Write the vertices of streamlines [s_begin, s_end) to the int32 buffer at
    xyz_ptr (host memory), at positions given by offsets (len s_end-s_begin+1)."""
    s_end = ss.n_streamlines if s_end is None else s_end
    vp, sp = vs._c(), ss._c()
    rl = np.ascontiguousarray(vols.roi_lin)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    assert len(off) == s_end - s_begin + 1
    lib().synth_fill(ctypes.byref(vp), ctypes.byref(sp), _ptr(rl), len(rl), s_begin, s_end,
                     _ptr(off), xyz_ptr, threads or n_threads())


def make_tractogram(vs: VolumeSpec, ss: StreamlineSpec, vols: Volumes, s_begin: int = 0,
                    s_end: int | None = None, threads: int | None = None) -> Tractogram:
    s_end = ss.n_streamlines if s_end is None else s_end
    counts = count_vertices(vs, ss, vols, s_begin, s_end, threads)
    offsets = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    xyz = np.empty((int(offsets[-1]), 3), dtype=np.int32)
    fill_vertices(vs, ss, vols, offsets, _ptr(xyz), s_begin, s_end, threads)
    return Tractogram(xyz, offsets)


# ------------------------------------------------------------------ presets

HCP_DIMS = (145, 174, 145)


def _thalami(dims, res_mm, scale=1.0):
    """Two thalamus-like ellipsoids at the brain centre +-12 mm in x, semi-axes
    (10, 16.25, 10) mm times scale, in voxel units."""
    c = [d / 2.0 for d in dims]
    off = 12.0 / res_mm
    ax = tuple(v * scale / res_mm for v in (10.0, 16.25, 10.0))
    return [(c[0] - off, c[1], c[2]), (c[0] + off, c[1], c[2])], [ax, ax]


def _brain(dims):
    return tuple(d / 2.0 for d in dims), tuple(0.42 * d for d in dims)


def volume_spec(cfg: int, subject: int = 0, **over) -> VolumeSpec:
    if cfg == 0:
        vs = VolumeSpec((32, 32, 32), (16.0, 16.0, 16.0), (15.0, 15.0, 15.0), 13.0 / 15.0, 8, 0,
                        [(16.0, 16.0, 16.0)], [(3.0, 4.0, 4.0)])
    elif cfg in (1, 4):
        bc, ba = _brain(HCP_DIMS)
        rc, ra = _thalami(HCP_DIMS, 1.25)
        vs = VolumeSpec(HCP_DIMS, bc, ba, 13.0 / 15.0, 70, 1 if cfg == 1 else 1000 + subject, rc, ra)
    elif cfg == 2:
        dims = (260, 311, 260)
        bc, ba = _brain(dims)
        rc, ra = _thalami(dims, 0.7)
        vs = VolumeSpec(dims, bc, ba, 13.0 / 15.0, 360, 2, rc, ra)
    elif cfg == 3:
        d = batched_subject_draws(subject)
        bc, ba = _brain(d["dims"])
        rc, ra = _thalami(d["dims"], 1.25, d["thal_scale"])
        vs = VolumeSpec(d["dims"], bc, ba, 13.0 / 15.0, d["M"], subject, rc, ra)
    else:
        raise ValueError(f"unknown config {cfg}")
    for k, v in over.items():
        setattr(vs, k, v)
    return vs


def streamline_spec(cfg: int, subject: int = 0, n_streamlines: int | None = None, **over) -> StreamlineSpec:
    if cfg == 0:
        ss = StreamlineSpec(20_000, seed=0, len_mode=0, len_a=20, len_b=120, res_mm=1.0)
    elif cfg == 1:
        ss = StreamlineSpec(2_000_000, seed=1, len_mode=1, len_a=80.0, len_sigma=0.5,
                            len_lo=20.0, len_hi=250.0, res_mm=1.25)
    elif cfg == 2:
        # mean 200 vertices at 0.35 mm per step: median = mean * exp(-sigma^2 / 2)
        ss = StreamlineSpec(5_000_000, seed=2, len_mode=1, len_a=200 * 0.35 * math.exp(-0.125),
                            len_sigma=0.5, len_lo=20.0, len_hi=250.0, res_mm=0.7)
    elif cfg == 3:
        d = batched_subject_draws(subject)
        ss = StreamlineSpec(d["ns"], seed=subject, subject=subject, len_mode=1, len_a=80.0,
                            len_sigma=0.5, len_lo=20.0, len_hi=250.0, res_mm=1.25)
    elif cfg == 4:
        ss = StreamlineSpec(2_000_000, seed=1000 + subject, subject=subject, len_mode=1, len_a=80.0,
                            len_sigma=0.5, len_lo=20.0, len_hi=250.0, res_mm=1.25)
    else:
        raise ValueError(f"unknown config {cfg}")
    if n_streamlines is not None:
        ss.n_streamlines = int(n_streamlines)
    for k, v in over.items():
        setattr(ss, k, v)
    return ss


def batched_subject_draws(subject: int) -> dict:
    """Per-subject shape of the 64-subject batch: grid axes uniform in
    [96, HCP dim], streamline count lognormal (median sqrt(5e4 * 2e6), sigma
    ln(40)/4) clipped to [5e4, 2e6], N uniform in [1,000, 12,000] (thalamus
    scaled to match at 1.25 mm), M uniform over {8, 70, 360}."""
    u = splitmix64(0xBA7C4ED0 + subject, 8).astype(np.float64) / 2.0**64
    dims = tuple(int(96 + min(int(u[a] * (HCP_DIMS[a] - 96 + 1)), HCP_DIMS[a] - 96)) for a in range(3))
    z = math.sqrt(-2.0 * math.log(max(u[3], 1e-300))) * math.cos(2.0 * math.pi * u[4])
    ns = math.exp(math.log(math.sqrt(5e4 * 2e6)) + (math.log(40.0) / 4.0) * z)
    ns = int(min(max(ns, 5e4), 2e6))
    n_target = 1000 + u[5] * 11000
    n_hcp = 2 * (4.0 / 3.0) * math.pi * 10.0 * 16.25 * 10.0 / 1.25**3
    M = (8, 70, 360)[min(int(u[6] * 3), 2)]
    return {"dims": dims, "ns": ns, "thal_scale": (n_target / n_hcp) ** (1.0 / 3.0), "M": M,
            "N_target": int(n_target)}


def make_subject(cfg: int, subject: int = 0, n_streamlines: int | None = None,
                 s_begin: int = 0, threads: int | None = None):
    """(Volumes, Tractogram) for a preset; n_streamlines truncates the preset's
    streamline count (the first n streamlines are the same as in the full set)."""
    vs = volume_spec(cfg, subject)
    ss = streamline_spec(cfg, subject)
    vols = make_volumes(vs, threads)
    n = ss.n_streamlines if n_streamlines is None else n_streamlines
    tract = make_tractogram(vs, ss, vols, s_begin, s_begin + n, threads)
    return vols, tract
