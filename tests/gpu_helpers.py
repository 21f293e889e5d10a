"""Shared helpers of the GPU tests: run the CUDA path through the C ABI."""
from __future__ import annotations

import numpy as np


def as_device(a: np.ndarray):
    import torch
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def run_gpu(roi, lab, dims, N, M, xyz, offsets, where: str = "device", options: dict | None = None,
            chunks: int = 1, ctx=None):
    """C, C_end (int32 numpy) and stats from the library.  where: 'device'
    (torch CUDA tensors), 'host' (numpy) or 'pinned' (page-locked torch)."""
    import torch
    from paper_2302_09247_gb300 import fastcod as fc

    own = ctx is None
    if own:
        ctx = fc.Context(0)
    try:
        for k, v in (options or {}).items():
            ctx.set_option(k, v)
        if where == "device":
            ctx.set_volumes(as_device(roi), as_device(lab), dims, N, M)
        else:
            ctx.set_volumes(np.ascontiguousarray(roi), np.ascontiguousarray(lab), dims, N, M)
        ns = len(offsets) - 1
        bounds = np.linspace(0, ns, chunks + 1).astype(np.int64)
        for c in range(chunks):
            b, e = int(bounds[c]), int(bounds[c + 1])
            o = np.ascontiguousarray(offsets[b:e + 1] - offsets[b])
            x = np.ascontiguousarray(xyz[offsets[b]:offsets[e]])
            if where == "device":
                ctx.add_streamlines(as_device(x), as_device(o))
                torch.cuda.synchronize()
            elif where == "pinned":
                xp = torch.from_numpy(x).pin_memory()
                op = torch.from_numpy(o).pin_memory()
                ctx.add_streamlines(xp, op)
                ctx.sync()
            else:
                ctx.add_streamlines(x, o)
        C = ctx.connectivity()
        Ce = ctx.endpoint_connectivity()
        st = ctx.stats()
        return C, Ce, st
    finally:
        if own:
            ctx.close()


def range_end_streamlines(rng, dims):
    """Streamlines (xyz int32 [n][3], offsets int64) with vertices exactly at
    -2^24 and 2^24 - 1, the ends of the accepted coordinate range: segments
    across the whole range on one, two and three axes, segments in an
    extreme plane, single vertices at corners, segments from the middle of
    the grid out to an extreme, and 40 ordinary short walks in the grid."""
    lo, hi = -(1 << 24), (1 << 24) - 1
    inside = [int(0.5 * d * 1024) for d in dims]
    lines = [
        [[lo, lo, lo], [hi, hi, hi]],                  # the main diagonal of the range
        [[hi, hi, hi], [lo, lo, lo]],                  # reversed
        [[lo, inside[1], inside[2]], [hi, inside[1], inside[2]]],  # one axis, through the grid
        [[lo, lo, inside[2]], [hi, hi, inside[2]]],    # two axes
        [[lo, hi, 512], [1000, 1000, hi]],             # mixed signs
        [[lo, 0, 0], [lo, 5 * 1024, 3 * 1024], [lo, 9 * 1024, 0]],  # in the plane x = -2^24
        [[hi, 7 * 1024, 2 * 1024], [hi, 8 * 1024, 2 * 1024]],      # in the plane x = 2^24 - 1
        [[lo, lo, lo]], [[hi, hi, hi]], [[lo, hi, lo]],  # single vertices at corners
        [inside, [hi, inside[1], inside[2]]],          # out of the grid to the top end
        [inside, [inside[0], lo, inside[2]]],          # and to the bottom end
        [[lo, lo, lo], inside, [hi, hi, hi]],          # in from one corner, out to the other
    ]
    for _ in range(40):  # ordinary short walks between them
        c = rng.uniform(0, 1, size=3) * np.array(dims) * 1024
        T = int(rng.integers(2, 30))
        lines.append((np.round(c) + np.cumsum(rng.integers(-512, 513, size=(T, 3)), axis=0)).astype(np.int64).tolist())
    counts = [len(v) for v in lines]
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    xyz = np.concatenate([np.asarray(v, dtype=np.int64).reshape(-1, 3) for v in lines]).astype(np.int32)
    return xyz, off
