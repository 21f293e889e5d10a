"""Small adversarial inputs: random volumes on tiny grids and streamlines whose
vertices are snapped to coarse lattices (multiples of 256/512/1024 units), so
that vertices on planes, edges and corners, segments lying in planes, zero-
length segments, T = 0 / T = 1 streamlines and points off the grid are
frequent.  Holds no connectivity arithmetic.
"""
from __future__ import annotations

import json
import os

import numpy as np

U = 1024


def random_volumes(rng: np.random.Generator, dims, n_roi: int, n_labels: int, p_roi: float = 0.25,
                   p_lab: float = 0.4, many_to_one: bool = False):
    """(roi int32 [Dz,Dy,Dx], lab uint16 [Dz,Dy,Dx], N, M)."""
    Dx, Dy, Dz = dims
    nvox = Dx * Dy * Dz
    roi = np.full(nvox, -1, dtype=np.int32)
    is_roi = rng.random(nvox) < p_roi
    k = int(is_roi.sum())
    if many_to_one:
        roi[is_roi] = rng.integers(0, max(n_roi, 1), size=k)
        N = n_roi
    else:
        roi[is_roi] = np.arange(k, dtype=np.int32)
        N = k
    lab = np.zeros(nvox, dtype=np.uint16)
    has = rng.random(nvox) < p_lab
    lab[has] = rng.integers(1, n_labels + 1, size=int(has.sum())).astype(np.uint16)
    return roi.reshape(Dz, Dy, Dx), lab.reshape(Dz, Dy, Dx), int(N), int(n_labels)


def random_streamlines(rng: np.random.Generator, dims, n: int, max_len: int = 12, margin: int = 2):
    """(xyz int32 [nv,3], offsets int64 [n+1]) with lattice-snapped vertices in
    [-margin, dim+margin) voxels, including T = 0 and T = 1 streamlines."""
    hi = np.array(dims, dtype=np.int64) + margin
    lo = -margin * np.ones(3, dtype=np.int64)
    pts, counts = [], []
    for _ in range(n):
        u = rng.random()
        T = 0 if u < 0.03 else (1 if u < 0.1 else int(rng.integers(2, max_len + 1)))
        snap = int((1, 256, 512, 1024)[rng.integers(4)])
        mode = rng.integers(3)
        v = np.empty((T, 3), dtype=np.int64)
        if T:
            v[0] = rng.integers(lo * U, hi * U)
        for t in range(1, T):
            if mode == 0:  # long jumps anywhere
                v[t] = rng.integers(lo * U, hi * U)
            else:  # short steps (about half a voxel), sometimes axis-aligned
                step = rng.integers(-700, 701, size=3)
                if rng.random() < 0.3:
                    step[rng.integers(3)] = 0
                v[t] = v[t - 1] + step
        if T and snap > 1:
            v = (v // snap) * snap
        pts.append(v)
        counts.append(T)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    xyz = np.concatenate(pts).astype(np.int32) if offsets[-1] else np.zeros((0, 3), dtype=np.int32)
    return xyz, offsets


def toy_fixture(path: str):
    """Volumes and streamlines of a tests/golden toy JSON fixture."""
    with open(path) as f:
        d = json.load(f)
    Dx, Dy, Dz = d["dims"]
    roi = np.full((Dz, Dy, Dx), -1, dtype=np.int32)
    lab = np.zeros((Dz, Dy, Dx), dtype=np.uint16)
    for name, (x, y, z) in d["roi_voxels"].items():
        roi[z, y, x] = int(name.split()[1])
    for name, vox in d["label_voxels"].items():
        for x, y, z in vox:
            lab[z, y, x] = int(name.split()[1])
    verts = [np.asarray(s["vertices"], dtype=np.int32).reshape(-1, 3) for s in d["streamlines"]]
    offsets = np.zeros(len(verts) + 1, dtype=np.int64)
    np.cumsum([len(v) for v in verts], out=offsets[1:])
    xyz = np.concatenate(verts).astype(np.int32)
    return d, roi, lab, xyz, offsets


GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")
